"""allegro_neighbors_noalloc (the entry point for callers that cannot allocate
device memory, e.g. under stream capture or inside an MD engine's own memory
pool) against the context path allegro_neighbors + allegro_get_neighbors:
identical (i, j, S) sets, on two calls in a row that share its fixed scratch.
Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_same_edges, lib_model
from synth import ARCHS, make_weights, weights_to_blob, lattice_box

pytestmark = pytest.mark.gpu


def _noalloc(L, pos_dev, cell, cap):
    import torch
    n = pos_dev.shape[0]
    i = torch.empty(cap, dtype=torch.int32, device="cuda")
    j = torch.empty(cap, dtype=torch.int32, device="cuda")
    S = torch.empty(cap, 3, dtype=torch.int32, device="cuda")
    ne = ctypes.c_int64(-1)
    cellh = np.ascontiguousarray(cell, dtype=np.float64)
    pbc = np.ones(3, np.uint8)
    st = L.allegro_neighbors_noalloc(pos_dev.data_ptr(), n, cellh.ctypes.data, pbc.ctypes.data, 4.0,
                                     i.data_ptr(), j.data_ptr(), S.data_ptr(), cap, ctypes.byref(ne), None)
    assert st == 0, st
    E = ne.value
    return i[:E].cpu().numpy(), j[:E].cpu().numpy(), S[:E].cpu().numpy()


def test_noalloc_matches_context_path_twice():
    import torch
    arch = ARCHS["c1"]
    m = lib_model(weights_to_blob(arch, make_weights(arch, 0)))
    from paper_2304_10061_gb300 import _lib
    L = _lib.load()
    boxes = [lattice_box(3000, (3000 / 0.1) ** (1 / 3), seed=21), lattice_box(800, (800 / 0.1) ** (1 / 3), seed=22)]
    for s in boxes:                                   # two calls in a row, different sizes
        pos = torch.tensor(s.pos, device="cuda")
        got = _noalloc(L, pos, s.cell, 40 * s.n_atoms)
        m.neighbors(s.pos, s.species % 2, s.cell)
        assert_same_edges(got, m.get_neighbors())
    m.close()


def test_noalloc_rejects_oversize_and_small_capacity():
    import torch
    from paper_2304_10061_gb300 import _lib
    L = _lib.load()
    pos = torch.zeros(16385, 3, dtype=torch.float64, device="cuda")
    ne = ctypes.c_int64(0)
    cell = np.eye(3) * 100.0
    assert L.allegro_neighbors_noalloc(pos.data_ptr(), 16385, cell.ctypes.data, None, 4.0, None, None, None, 0,
                                       ctypes.byref(ne), None) == 4
    s = lattice_box(500, (500 / 0.1) ** (1 / 3), seed=3)
    pd = torch.tensor(s.pos, device="cuda")
    assert L.allegro_neighbors_noalloc(pd.data_ptr(), 500, s.cell.ctypes.data, None, 4.0, None, None, None, 0,
                                       ctypes.byref(ne), None) == 4
    assert ne.value > 0                              # the needed count is still reported
