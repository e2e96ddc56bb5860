"""ctypes binding of liballegro_gb300.so: the same entry points as include/allegro.h.

Argument marshalling only; every step of the computation runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "liballegro_gb300.so")

ALLEGRO_OK = 0
STATUS_NAMES = {
    0: "ALLEGRO_OK", 1: "ALLEGRO_E_INVALID", 2: "ALLEGRO_E_OOM", 3: "ALLEGRO_E_CUDA",
    4: "ALLEGRO_E_CAPACITY", 5: "ALLEGRO_E_TIMEOUT", 6: "ALLEGRO_E_NONFINITE", 7: "ALLEGRO_E_STATE",
}
PREC = {"fp32": 0, "bf16": 1, "tf32": 2, "fp8": 3}

EXPORTS = ("allegro_create", "allegro_set_stream", "allegro_set_pair_cutoffs", "allegro_set_zbl", "allegro_reserve", "allegro_neighbors",
           "allegro_neighbors_batched", "allegro_energy_forces", "allegro_get_neighbors",
           "allegro_profile", "allegro_profile_report", "allegro_neighbors_noalloc", "allegro_md_verlet", "allegro_set_md_skin", "allegro_md_rebuilds",
           "allegro_set_autotune", "allegro_set_graphs", "allegro_autotune_report", "allegro_list_size",
           "allegro_neighbors_local",
           "allegro_last_error",
           "allegro_destroy")

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (once) and declare its prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i32, i64, sz, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
    L.allegro_create.argtypes = [vp, sz, vp, i32, ctypes.c_double, i32, i32, ctypes.POINTER(vp)]
    L.allegro_set_stream.argtypes = [vp, vp]
    L.allegro_reserve.argtypes = [vp, i64, i64, i32, i64]
    L.allegro_set_pair_cutoffs.argtypes = [vp, dp, i32]
    L.allegro_set_zbl.argtypes = [vp, dp, i32]
    L.allegro_neighbors.argtypes = [vp, i64, dp, dp, dp, dp, ctypes.POINTER(i64)]
    L.allegro_neighbors_batched.argtypes = [vp, i32, dp, dp, dp, dp, dp, ctypes.POINTER(i64)]
    L.allegro_neighbors_local.argtypes = [vp, i64, i64, dp, dp, dp, dp, ctypes.POINTER(i64)]
    L.allegro_energy_forces.argtypes = [vp, dp, dp, dp, dp]
    L.allegro_get_neighbors.argtypes = [vp, dp, dp, dp, i64]
    L.allegro_profile.argtypes = [vp, i32]
    L.allegro_profile_report.argtypes = [vp, ctypes.c_char_p, sz, ctypes.POINTER(i64)]
    L.allegro_neighbors_noalloc.argtypes = [dp, i64, dp, dp, ctypes.c_double, dp, dp, dp, i64,
                                            ctypes.POINTER(i64), vp]
    L.allegro_md_verlet.argtypes = [vp, i64, dp, dp, dp, dp, i32, dp, dp, ctypes.c_double, i64, dp, dp]
    L.allegro_set_md_skin.argtypes = [vp, ctypes.c_double]
    L.allegro_set_autotune.argtypes = [vp, i32]
    L.allegro_list_size.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]
    L.allegro_set_graphs.argtypes = [vp, i32]
    L.allegro_autotune_report.argtypes = [vp, ctypes.c_char_p, sz]
    L.allegro_md_rebuilds.argtypes = [vp, ctypes.POINTER(i64)]
    L.allegro_last_error.argtypes = [vp]
    L.allegro_last_error.restype = ctypes.c_char_p
    L.allegro_destroy.argtypes = [vp]
    L.allegro_destroy.restype = None
    for name in EXPORTS:
        if name not in ("allegro_last_error", "allegro_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L
