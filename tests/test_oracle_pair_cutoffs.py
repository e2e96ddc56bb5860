"""Pins of the oracle's per-ordered-species-pair cutoffs (Sec. "Species-dependent
cutoffs"; the production values in "Training details"): the neighbour rule
against its brute-force definition, the ordering of a pair, the reduction to
the single-cutoff model, the inertness of edges beyond their pair's cutoff (the
basis and envelope take the pair's cutoff), continuity across a pair cutoff,
forces against finite differences, O(3) invariance, and the edge count of the
water-density box against the uniform-density expectation (no GPU)."""
from dataclasses import replace

import numpy as np
import pytest

from oracle.allegro import AllegroOracle
from oracle.neighbors import brute_force, neighbor_list
from synth import Arch, SPECIES_NAMES, WATER_MIX, lattice_box, make_weights, paper_pair_cutoffs

H, O, C, N, S_ = (SPECIES_NAMES.index(x) for x in ("H", "O", "C", "N", "S"))
TABLE = paper_pair_cutoffs()
ARCH = Arch(n_species=5, lmax=1, n_layers=2, channels=4, two_body=(16,), latent=(16,), edge=(8,),
            pair_rc=TABLE)


@pytest.fixture(scope="module")
def model():
    return AllegroOracle(ARCH, make_weights(ARCH, 11))


def _edges(s, pair_rc=TABLE, r_c=4.0):
    return neighbor_list(s.pos, s.cell, s.pbc, r_c, species=s.species, pair_rc=pair_rc)


def _ef(model, s, edges=None, pos=None, cell="same"):
    pos = s.pos if pos is None else pos
    cell = s.cell if isinstance(cell, str) else cell
    if edges is None:
        edges = neighbor_list(pos, cell, s.pbc, 4.0, species=s.species, pair_rc=model.arch.pair_rc)
    i, j, S = edges
    return model.energy_forces(pos, s.species, cell, i, j, S)


def _box(n=48, seed=5):
    return lattice_box(n, (n / 0.1) ** (1 / 3), seed=seed)


def test_paper_table_values_and_order():
    t = np.asarray(TABLE)
    assert t[H, H] == 3.0 and t[O, H] == 3.0
    assert t[H, C] == 1.25 and t[H, O] == 1.25
    assert t[C, H] == 4.0 and t[O, O] == 4.0 and t[N, S_] == 4.0
    assert int((t != 4.0).sum()) == 4


def test_pair_rule_matches_brute_force():
    for seed, n in [(1, 30), (2, 64)]:
        s = lattice_box(n, (n / 0.1) ** (1 / 3), seed=seed, jitter=0.45)
        ref = brute_force(s.pos, s.cell, s.pbc, 4.0, species=s.species, pair_rc=TABLE)
        got = _edges(s)
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
        # and it is a strict subset of the single-cutoff list
        full = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
        assert 0 < ref[0].size < full[0].size


def test_pairs_are_ordered():
    # an H centre and a C neighbour 2 A apart: C-H (4.0) is an edge, H-C (1.25) is not
    pos = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    species = np.array([H, C])
    i, j, S = brute_force(pos, None, [False] * 3, 4.0, species=species, pair_rc=TABLE)
    assert list(zip(i.tolist(), j.tolist())) == [(1, 0)]
    # inside 1.25 A both directions exist
    i, j, S = brute_force(pos * 0.6, None, [False] * 3, 4.0, species=species, pair_rc=TABLE)
    assert sorted(zip(i.tolist(), j.tolist())) == [(0, 1), (1, 0)]


def test_uniform_table_is_the_single_cutoff_model():
    s = _box()
    flat = tuple(tuple(4.0 for _ in range(5)) for _ in range(5))
    w = make_weights(ARCH, 11)
    m_tab = AllegroOracle(replace(ARCH, pair_rc=flat), w)
    m_one = AllegroOracle(replace(ARCH, pair_rc=None), w)
    e_one = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    e_tab = _edges(s, pair_rc=flat)
    for a, b in zip(e_one, e_tab):
        np.testing.assert_array_equal(a, b)
    E1, Ea1, F1, W1 = m_one.energy_forces(s.pos, s.species, s.cell, *e_one)
    E2, Ea2, F2, W2 = m_tab.energy_forces(s.pos, s.species, s.cell, *e_tab)
    assert abs(E1 - E2) <= 1e-12 * abs(E1)
    np.testing.assert_allclose(F2, F1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(W2, W1, rtol=0, atol=1e-11)


def test_edges_beyond_their_pair_cutoff_are_inert(model):
    # the single-cutoff candidate list holds pairs beyond their pair's cutoff; the
    # envelope and basis of each edge take its pair's cutoff, so they add nothing
    s = _box()
    full = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    E1, Ea1, F1, W1 = _ef(model, s, edges=full)
    E2, Ea2, F2, W2 = _ef(model, s)
    assert abs(E1 - E2) <= 1e-12 * abs(E1)
    np.testing.assert_allclose(Ea1, Ea2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(F1, F2, rtol=0, atol=1e-12)


def test_energy_continuous_across_a_pair_cutoff(model):
    # H, O and a C spectator; the H-O distance crosses the H-O cutoff (1.25 A);
    # the O-H edge (3.0 A) stays
    def energy(r):
        pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [0.3, 1.7, 0.4]])
        s = type("S", (), {})()
        s.pos, s.species, s.cell, s.pbc = pos, np.array([H, O, C]), None, [False] * 3
        return _ef(model, s)[0]
    rc = TABLE[H][O]
    h = 1e-4
    # second difference across the cutoff: O(h^2) for a smooth energy, O(jump) otherwise
    # (an envelope on the single 4 A cutoff would leave the H-O edge a finite jump here)
    d2 = energy(rc - h) - 2.0 * energy(rc + h) + energy(rc + 3 * h)
    assert abs(d2) < 1e-6, d2
    assert abs(energy(rc + 0.05) - energy(rc + h)) > 1e-5   # the energy does depend on r there


def test_forces_match_finite_differences(model):
    s = _box(40, seed=8)
    E, Ea, F, W = _ef(model, s)
    rng = np.random.default_rng(3)
    h = 1e-5
    for a in rng.choice(s.pos.shape[0], 4, replace=False):
        for x in range(3):
            p1 = s.pos.copy(); p1[a, x] += h
            p0 = s.pos.copy(); p0[a, x] -= h
            fd = -(_ef(model, s, pos=p1)[0] - _ef(model, s, pos=p0)[0]) / (2 * h)
            assert abs(fd - F[a, x]) <= 1e-6 * max(1.0, np.abs(F).max()), (a, x, fd, F[a, x])


def test_rotation_reflection_invariance(model):
    s = _box(40, seed=9)
    E, Ea, F, W = _ef(model, s)
    q, _ = np.linalg.qr(np.random.default_rng(4).normal(size=(3, 3)))
    R = -q
    E2, Ea2, F2, W2 = _ef(model, s, pos=s.pos @ R.T, cell=s.cell @ R.T)
    assert abs(E - E2) < 1e-10 * abs(E)
    np.testing.assert_allclose(F2, F @ R.T, atol=1e-10)
    np.testing.assert_allclose(W2, R @ W @ R.T, atol=1e-9)


def test_edge_count_on_the_water_density_box():
    # uniform density rho: an ordered (a, b) pair count ~ N x_a x_b rho (4/3) pi rc_ab^3,
    # so the table keeps sum_ab x_a x_b (rc_ab / 4)^3 of the single-cutoff edges; the
    # jittered lattice has no pairs closer than ~1.07 A, which moves the short (1.25 A)
    # entries, a small share
    n = 4096
    s = lattice_box(n, (n / 0.1) ** (1 / 3), seed=3)
    full = neighbor_list(s.pos, s.cell, s.pbc, 4.0)[0].size
    tab = _edges(s)[0].size
    x = np.bincount(s.species, minlength=5) / n
    t = np.asarray(TABLE)
    expect = float((x[:, None] * x[None, :] * (t / 4.0) ** 3).sum())
    frac = tab / full
    assert abs(frac - expect) < 0.05 * expect, (frac, expect)
    assert 1.9 < full / tab < 2.6   # about 2.2x fewer edges for this composition
