"""Helpers shared by the GPU tests: build/load the library, run it through the
C ABI binding, and compare with the oracle."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# FP32 path (the benchmark spec): per-atom energy rel 1e-5 (scale max(|E_i|, rms E_i)), max |dF| <= 1e-4 rms|F|
FP32_E, FP32_F, FP32_W = 1e-5, 1e-4, 1e-5
# BF16 MLP path: force RMS error <= 2 % of RMS|F|
BF16_F_RMS = 2e-2


def lib_model(blob, precision="fp32", **kw):
    import __graft_entry__ as g
    g.build()
    from paper_2304_10061_gb300 import Allegro
    return Allegro(blob, precision=precision, **kw)


def sorted_edges(i, j, S):
    i = np.asarray(i, np.int64); j = np.asarray(j, np.int64); S = np.asarray(S, np.int64).reshape(-1, 3)
    a = np.lexsort((S[:, 2], S[:, 1], S[:, 0], j, i))
    return i[a], j[a], S[a]


def assert_same_edges(got, want):
    gi, gj, gS = sorted_edges(*got)
    wi, wj, wS = sorted_edges(*want)
    assert len(gi) == len(wi), (len(gi), len(wi))
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gj, wj)
    np.testing.assert_array_equal(gS, wS)


def errors(Ea, F, W, Ea0, F0, W0):
    scale = np.maximum(np.abs(Ea0), np.sqrt((Ea0 ** 2).mean()))
    rms = np.sqrt((F0 ** 2).mean()) if F0.size else 1.0
    out = dict(e_rel=float(np.max(np.abs(Ea - Ea0) / scale)) if Ea0.size else 0.0,
               f_max=float(np.abs(F - F0).max() / rms) if F0.size else 0.0,
               f_rms=float(np.sqrt(((F - F0) ** 2).mean()) / rms) if F0.size else 0.0)
    if W is not None:
        out["w_rel"] = float(np.abs(W - W0).max() / max(np.abs(W0).max(), 1e-300))
    return out
