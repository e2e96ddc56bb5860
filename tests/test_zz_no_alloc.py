"""allegro_neighbors_noalloc: the neighbour search for callers that cannot
allocate device memory while they run (an MD engine whose own pool allocator
owns the GPU's memory, a steady-state loop with a fixed footprint), whose
scratch is one fixed device array inside the library.

Checked against the context path (allegro_neighbors + allegro_get_neighbors)
on two calls in a row that share the scratch, and against the oracle's
brute-force pair rule on triclinic, mixed-periodicity, non-periodic,
unwrapped and empty inputs and on a non-default stream; plus the input checks
that reject work the fixed scratch or the launch cannot take.  Collected last
on purpose, so that a run stopping at its first failure has run the rest."""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_same_edges, lib_model
from oracle.neighbors import brute_force
from synth import ARCHS, make_weights, weights_to_blob, lattice_box

pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as g
    g.build()
    from paper_2304_10061_gb300 import _lib as lb
    return lb.load()


def _noalloc(L, pos, cell, pbc, cap, r_c=4.0, stream=None):
    """Runs the entry point on device copies of `pos`; returns (status, edges or None)."""
    import torch
    n = len(pos)
    pd = torch.tensor(np.asarray(pos, np.float64).reshape(-1, 3), device="cuda")
    i = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    j = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    S = torch.full((max(cap, 1), 3), -7, dtype=torch.int32, device="cuda")
    ne = ctypes.c_int64(-1)
    cellh = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
    pbch = None if pbc is None else np.ascontiguousarray(pbc, dtype=np.uint8)
    st = L.allegro_neighbors_noalloc(pd.data_ptr() if n else None, n,
                                     None if cellh is None else cellh.ctypes.data,
                                     None if pbch is None else pbch.ctypes.data, float(r_c),
                                     i.data_ptr(), j.data_ptr(), S.data_ptr(), cap, ctypes.byref(ne),
                                     None if stream is None else ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        return st, ne.value, None
    E = ne.value
    return st, E, (i[:E].cpu().numpy(), j[:E].cpu().numpy(), S[:E].cpu().numpy())


def test_noalloc_matches_context_path_twice():
    arch = ARCHS["c1"]
    m = lib_model(weights_to_blob(arch, make_weights(arch, 0)))
    L = _lib()
    boxes = [lattice_box(3000, (3000 / 0.1) ** (1 / 3), seed=21), lattice_box(800, (800 / 0.1) ** (1 / 3), seed=22)]
    for s in boxes:                                   # two calls in a row, different sizes
        st, _, got = _noalloc(L, s.pos, s.cell, None, 40 * s.n_atoms)
        assert st == 0, st
        m.neighbors(s.pos, s.species % 2, s.cell)
        assert_same_edges(got, m.get_neighbors())
    m.close()


TRICLINIC = np.array([[6.0, 0.0, 0.0], [2.1, 5.5, 0.0], [-1.3, 1.7, 7.2]])


@pytest.mark.parametrize("case", ["triclinic_pbc", "mixed_110", "mixed_101", "no_cell", "shift_-0.4",
                                  "shift_+1.4", "unwrapped_+2", "thin_cell"])
def test_noalloc_matches_brute_force(case):
    L = _lib()
    rng = np.random.default_rng(11)
    cell, pbc = TRICLINIC, [1, 1, 1]
    frac = rng.uniform(0.0, 1.0, (60, 3))
    if case == "mixed_110":
        pbc = [1, 1, 0]
    elif case == "mixed_101":
        pbc = [1, 0, 1]
    elif case == "no_cell":
        cell, pbc = None, None
    elif case == "shift_-0.4":
        frac[:20] -= 0.4                              # near the old [-0.5, 1.5) edge
    elif case == "shift_+1.4":
        frac[:20] += 1.4
    elif case == "unwrapped_+2":
        frac[:7, 1] += 2.0                            # atoms two cells out along b
        frac[7:9, 0] -= 3.0
    elif case == "thin_cell":
        cell = np.diag([2.5, 3.0, 9.0])               # periodic self-images within the cutoff
        frac = rng.uniform(0.0, 1.0, (6, 3))
    base = TRICLINIC if cell is None else cell
    pos = frac @ base
    st, E, got = _noalloc(L, pos, cell, pbc, 100000)
    assert st == 0, st
    want = brute_force(pos, cell, [False] * 3 if pbc is None and cell is None else
                       ([True] * 3 if pbc is None else [bool(x) for x in pbc]), 4.0)
    assert_same_edges(got, want)
    if case == "thin_cell":
        i, j, S = got
        assert np.any((i == j) & np.any(S != 0, axis=1))


def test_noalloc_empty_and_single():
    L = _lib()
    st, E, got = _noalloc(L, np.zeros((0, 3)), np.eye(3) * 10, None, 0)
    assert st == 0 and E == 0
    st, E, got = _noalloc(L, np.array([[0.5, 0.5, 0.5]]), np.eye(3) * 3.0, None, 16)
    assert st == 0 and E == 6                         # the six nearest periodic images at 3.0 A


def test_noalloc_on_a_torch_stream():
    import torch
    L = _lib()
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=31)
    side = torch.cuda.Stream()
    st, E, got = _noalloc(L, s.pos, s.cell, None, 40000, stream=side)
    assert st == 0
    assert_same_edges(got, brute_force(s.pos, s.cell, [True] * 3, 4.0))


def test_noalloc_rejects_bad_inputs_without_damage():
    import torch
    L = _lib()
    ne = ctypes.c_int64(0)
    cell = np.eye(3) * 100.0
    pos = torch.zeros(16385, 3, dtype=torch.float64, device="cuda")
    # more atoms than the fixed scratch holds: rejected before any launch
    assert L.allegro_neighbors_noalloc(pos.data_ptr(), 16385, cell.ctypes.data, None, 4.0, None, None, None, 0,
                                       ctypes.byref(ne), None) == 4
    # non-finite or oversized cutoffs
    for rc in (float("inf"), float("nan"), 0.0, 401.0):
        assert L.allegro_neighbors_noalloc(pos.data_ptr(), 10, cell.ctypes.data, None, rc, None, None, None, 0,
                                           ctypes.byref(ne), None) == 1, rc
    # a non-finite position
    s = lattice_box(500, (500 / 0.1) ** (1 / 3), seed=3)
    p = s.pos.copy()
    p[17, 1] = np.nan
    st, _, _ = _noalloc(L, p, s.cell, None, 40000)
    assert st == 1
    # too small an output capacity: the needed count is still reported, outputs untouched
    st, E, _ = _noalloc(L, s.pos, s.cell, None, 0)
    assert st == 4 and E > 0
    st, E2, got = _noalloc(L, s.pos, s.cell, None, E)
    assert st == 0 and E2 == E
    assert_same_edges(got, brute_force(s.pos, s.cell, [True] * 3, 4.0))
