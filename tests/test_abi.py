"""The C-ABI library builds, loads and exports every entry point include/allegro.h
declares (no GPU needed; no compute calls)."""
import os
import re
import ctypes

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "allegro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(allegro_[a-z_]+)\s*\(", src)))


def test_build_and_exports():
    import __graft_entry__ as g
    g.build()
    from paper_2304_10061_gb300 import _lib
    L = _lib.load()
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.EXPORTS)


def test_status_codes_match_header():
    from paper_2304_10061_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "allegro.h")).read()
    for code, name in _lib.STATUS_NAMES.items():
        assert re.search(rf"\b{name}\s*=\s*{code}\b", src), name
    assert re.search(r"ALLEGRO_PREC_FP32\s*=\s*0", src) and re.search(r"ALLEGRO_PREC_BF16\s*=\s*1", src)


def test_null_arguments_rejected_without_gpu():
    """Argument checks that run before any device work."""
    from paper_2304_10061_gb300 import _lib
    L = _lib.load()
    out = ctypes.c_void_p()
    assert L.allegro_create(None, 0, None, 0, 0.0, 0, 0, ctypes.byref(out)) == 1
    assert L.allegro_energy_forces(None, None, None, None, None) == 1
    assert L.allegro_set_pair_cutoffs(None, None, 0) == 1
    assert L.allegro_last_error(None) == b"null context"
    L.allegro_destroy(None)


def test_weights_blob_roundtrip():
    from synth import ARCHS, make_weights, weights_to_blob, blob_to_weights
    for name, arch in ARCHS.items():
        w = make_weights(arch, 1)
        a2, w2 = blob_to_weights(weights_to_blob(arch, w))
        assert a2 == arch
        for k in w:
            np.testing.assert_array_equal(w[k], w2[k])


def test_oracle_not_imported_by_product():
    """The product path (package, bench's GPU leg) never reaches the oracle."""
    pkg = os.path.join(ROOT, "paper_2304_10061_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dp, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", src), f
