"""Pins of the oracle's neighbour rule: brute force is the definition; the
pruned search must equal it; hand-enumerated cases; pair symmetry."""
import os

import numpy as np
import pytest

from oracle.neighbors import brute_force, neighbor_list
from synth import random_box, lattice_box, molecule_batch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_golden_dimer_strict_cutoff():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "neighbors_dimer.txt")) if l[0] in "AB"]
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    cell = np.eye(3) * 5.0
    for case, rc in (("A", 4.0), ("B", 4.5)):
        exp = np.array([[int(v) for v in r[1:]] for r in rows if r[0] == case])
        for fn in (brute_force, neighbor_list):
            i, j, S = fn(pos, cell, [True] * 3, rc)
            got = np.concatenate([i[:, None], j[:, None], S], 1)
            np.testing.assert_array_equal(got, exp)


def test_pruned_equals_brute_force_random_box():
    s = random_box(64, 8.62, seed=0)
    assert _same(brute_force(s.pos, s.cell, s.pbc, 4.0), neighbor_list(s.pos, s.cell, s.pbc, 4.0))


def test_pruned_equals_brute_force_triclinic_and_small_cells():
    rng = np.random.default_rng(5)
    cell = np.array([[6.0, 0.0, 0.0], [2.1, 5.5, 0.0], [-1.3, 1.7, 7.2]])
    frac = rng.uniform(-0.2, 1.2, size=(40, 3))          # some atoms outside the cell
    pos = frac @ cell
    for pbc in ([True] * 3, [True, False, True], [False] * 3):
        assert _same(brute_force(pos, cell, pbc, 4.0), neighbor_list(pos, cell, pbc, 4.0))
    # cell thinner than r_c: many periodic self-images
    cell = np.diag([2.5, 3.0, 9.0])
    pos = rng.uniform(0, 1, size=(5, 3)) @ cell
    bf = brute_force(pos, cell, [True] * 3, 4.0)
    assert _same(bf, neighbor_list(pos, cell, [True] * 3, 4.0))
    assert np.any((bf[0] == bf[1]) & np.any(bf[2] != 0, axis=1))    # self-images present


def test_pruned_equals_brute_force_lattice_and_molecule():
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=9)
    assert _same(brute_force(s.pos, s.cell, s.pbc, 4.0), neighbor_list(s.pos, s.cell, s.pbc, 4.0))
    m = molecule_batch(3, seed=4)[2]
    assert _same(brute_force(m.pos, None, m.pbc, 4.0), neighbor_list(m.pos, None, m.pbc, 4.0))


def test_pair_symmetry_and_density():
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=3)
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    fwd = set(zip(i.tolist(), j.tolist(), map(tuple, S.tolist())))
    rev = set(zip(j.tolist(), i.tolist(), map(tuple, (-S).tolist())))
    assert fwd == rev
    mean = len(i) / 1000
    assert abs(mean - 0.1 * 4 / 3 * np.pi * 64) < 1.5          # ~26.8 neighbours at water density
    # self pair (i, i, 0) never present
    assert not np.any((i == j) & np.all(S == 0, axis=1))


def test_centers_subset_matches_full_rows():
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=3)
    full = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    cs = np.array([0, 17, 500, 999])
    sub = neighbor_list(s.pos, s.cell, s.pbc, 4.0, centers=cs)
    m = np.isin(full[0], cs)
    assert _same(sub, tuple(x[m] for x in full))


def test_unwrapped_positions_find_all_images():
    """Atoms outside the cell: the edge set equals that of the wrapped positions
    with the image shifts adjusted by the wrap counts."""
    rng = np.random.default_rng(5)
    cell = np.array([[6.0, 0.0, 0.0], [2.1, 5.5, 0.0], [-1.3, 1.7, 7.2]])
    frac = rng.uniform(-0.2, 1.2, size=(40, 3))
    w = np.floor(frac)
    pos = frac @ cell
    posw = (frac - w) @ cell
    i, j, S = neighbor_list(pos, cell, [True] * 3, 4.0)
    iw, jw, Sw = neighbor_list(posw, cell, [True] * 3, 4.0)
    # d = pos_j + S cell - pos_i = posw_j + (S + w_j - w_i) cell - posw_i
    a = set(zip(i.tolist(), j.tolist(), map(tuple, (S + w[j].astype(int) - w[i].astype(int)).tolist())))
    b = set(zip(iw.tolist(), jw.tolist(), map(tuple, Sw.tolist())))
    assert a == b
