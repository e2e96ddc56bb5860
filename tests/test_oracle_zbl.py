"""Pins of the oracle's ZBL repulsion (the production potential's repulsive term,
Sec. "Training details"; the readings are stated in oracle/zbl.py): the Coulomb
constant and the Bohr radius against their SI definitions, the screening
function's value at contact, the bare-Coulomb short-range limit, a repulsive and
monotone pair energy, the half-per-ordered-edge assembly with each edge's
envelope (uniform and per-pair cutoffs), forces against finite differences and
O(3) invariance with the term on (no GPU)."""
import math
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import zbl
from oracle.allegro import AllegroOracle, envelope
from oracle.neighbors import neighbor_list
from synth import Arch, SPECIES_NAMES, SPECIES_Z, lattice_box, make_weights, paper_pair_cutoffs

H, O = SPECIES_NAMES.index("H"), SPECIES_NAMES.index("O")
ARCH = Arch(n_species=5, lmax=1, n_layers=2, channels=4, two_body=(16,), latent=(16,), edge=(8,),
            zbl_z=SPECIES_Z)


@pytest.fixture(scope="module")
def weights():
    return make_weights(ARCH, 31)


def test_constants_from_si():
    e, eps0, hbar, me = 1.602176634e-19, 8.8541878128e-12, 1.054571817e-34, 9.1093837015e-31
    ke = e / (4 * math.pi * eps0) * 1e10           # e^2 / (4 pi eps0) in eV A
    a0 = 4 * math.pi * eps0 * hbar ** 2 / (me * e ** 2) * 1e10
    assert abs(zbl.KE - ke) < 1e-5
    assert abs(zbl.A0 - a0) < 1e-6


def test_screening_at_contact_and_coulomb_limit():
    assert abs(float(zbl.screening(torch.zeros(1, dtype=torch.float64))) - 1.0) < 1e-12
    for za, zb in [(1, 1), (8, 6), (16, 7)]:
        r = torch.tensor([1e-6], dtype=torch.float64)
        e = zbl.pair_energy(r, torch.tensor([za]), torch.tensor([zb]))
        assert abs(float(e * r) / (zbl.KE * za * zb) - 1.0) < 1e-4


def test_pair_energy_repulsive_and_monotone():
    r = torch.linspace(0.05, 4.0, 400, dtype=torch.float64)
    for za, zb in [(1, 1), (1, 8), (8, 8), (6, 16)]:
        e = zbl.pair_energy(r, torch.full_like(r, za), torch.full_like(r, zb))
        assert bool((e > 0).all())
        assert bool((e[1:] < e[:-1]).all())


def _pair(r, sa, sb):
    class S:
        pass
    s = S()
    s.pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    s.species = np.array([sa, sb])
    s.cell, s.pbc = None, [False] * 3
    return s


def _E(model, s):
    a = model.arch
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, a.r_c, species=s.species, pair_rc=a.pair_rc) \
        if a.pair_rc is not None else neighbor_list(s.pos, s.cell, s.pbc, a.r_c)
    return model.energy_forces(s.pos, s.species, s.cell, i, j, S)


@pytest.mark.parametrize("pair_table", [False, True])
def test_dimer_adds_half_per_ordered_edge(weights, pair_table):
    table = paper_pair_cutoffs() if pair_table else None
    on = AllegroOracle(replace(ARCH, pair_rc=table), weights)
    off = AllegroOracle(replace(ARCH, pair_rc=table, zbl_z=None), weights)
    r = 1.0
    s = _pair(r, H, O)
    E1, Ea1, _, _ = _E(on, s)
    E0, Ea0, _, _ = _E(off, s)
    rr = torch.tensor([r], dtype=torch.float64)
    pe = float(zbl.pair_energy(rr, torch.tensor([SPECIES_Z[H]]), torch.tensor([SPECIES_Z[O]])))
    rc_ho = table[H][O] if pair_table else 4.0
    rc_oh = table[O][H] if pair_table else 4.0
    u_ho = float(envelope(rr / rc_ho, ARCH.p_env))
    u_oh = float(envelope(rr / rc_oh, ARCH.p_env))
    # per atom: half the pair energy with that atom's ordered edge envelope, unscaled by sigma
    assert abs((Ea1[0] - Ea0[0]) - 0.5 * pe * u_ho) < 1e-10 * pe
    assert abs((Ea1[1] - Ea0[1]) - 0.5 * pe * u_oh) < 1e-10 * pe
    assert abs((E1 - E0) - 0.5 * pe * (u_ho + u_oh)) < 1e-10 * pe


def _box(n=40, seed=6):
    return lattice_box(n, (n / 0.1) ** (1 / 3), seed=seed)


def test_forces_match_finite_differences(weights):
    m = AllegroOracle(ARCH, weights)
    s = _box()
    E, Ea, F, W = _E(m, s)
    rng = np.random.default_rng(2)
    h = 1e-5
    for a in rng.choice(s.pos.shape[0], 4, replace=False):
        for x in range(3):
            p1 = s.pos.copy(); p1[a, x] += h
            p0 = s.pos.copy(); p0[a, x] -= h
            s1 = _box(); s1.pos = p1
            s0 = _box(); s0.pos = p0
            fd = -(_E(m, s1)[0] - _E(m, s0)[0]) / (2 * h)
            assert abs(fd - F[a, x]) <= 1e-6 * max(1.0, np.abs(F).max()), (a, x, fd, F[a, x])


def test_rotation_invariance(weights):
    m = AllegroOracle(ARCH, weights)
    s = _box(seed=7)
    E, Ea, F, W = _E(m, s)
    q, _ = np.linalg.qr(np.random.default_rng(5).normal(size=(3, 3)))
    s2 = _box(seed=7)
    s2.pos, s2.cell = s.pos @ q.T, s.cell @ q.T
    E2, Ea2, F2, W2 = _E(m, s2)
    assert abs(E - E2) < 1e-10 * abs(E)
    np.testing.assert_allclose(F2, F @ q.T, atol=1e-9)
    np.testing.assert_allclose(W2, q @ W @ q.T, atol=1e-8)
