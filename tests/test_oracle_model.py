"""Pins of the FP64 oracle model: symmetry, locality, derivatives, closed forms
and the bilinearity identity of Eq. 1 (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import so3
from oracle.allegro import AllegroOracle, bessel, envelope
from oracle.neighbors import neighbor_list
from oracle.verlet import verlet_step, kinetic_energy
from synth import Arch, make_weights, random_box, lattice_box, molecule_batch, make_config, SPECIES_MASSES

TINY = Arch(n_species=3, lmax=2, n_layers=2, channels=4, two_body=(16,), latent=(16,), edge=(8,))


def _system(n=40, seed=2):
    s = lattice_box(n, (n / 0.1) ** (1 / 3), seed=seed)
    s.species = s.species % 3
    return s


def _ef(model, s, pos=None, cell="same"):
    pos = s.pos if pos is None else pos
    cell = s.cell if isinstance(cell, str) else cell
    i, j, S = neighbor_list(pos, cell, s.pbc, model.arch.r_c)
    return model.energy_forces(pos, s.species, cell, i, j, S)


@pytest.fixture(scope="module")
def tiny():
    return AllegroOracle(TINY, make_weights(TINY, 3))


def _orth(seed, reflect):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return -q if reflect else q


@pytest.mark.parametrize("reflect", [False, True])
def test_rotation_reflection_invariance(tiny, reflect):
    s = _system()
    E, Ea, F, W = _ef(tiny, s)
    R = _orth(4, reflect)
    E2, Ea2, F2, W2 = _ef(tiny, s, pos=s.pos @ R.T, cell=s.cell @ R.T)
    assert abs(E - E2) < 1e-10 * abs(E)
    np.testing.assert_allclose(Ea2, Ea, atol=1e-10)
    np.testing.assert_allclose(F2, F @ R.T, atol=1e-10)
    np.testing.assert_allclose(W2, R @ W @ R.T, atol=1e-9)


def test_translation_and_permutation(tiny):
    s = _system()
    E, Ea, F, _ = _ef(tiny, s)
    E2, Ea2, F2, _ = _ef(tiny, s, pos=s.pos + np.array([0.37, -1.2, 5.1]))
    assert abs(E - E2) < 1e-10 * abs(E)
    np.testing.assert_allclose(F2, F, atol=1e-10)
    perm = np.random.default_rng(0).permutation(s.n_atoms)
    s.pos, s.species = s.pos[perm], s.species[perm]
    E3, Ea3, F3, _ = _ef(tiny, s)
    assert abs(E - E3) < 1e-10 * abs(E)
    np.testing.assert_allclose(Ea3, Ea[perm], atol=1e-10)
    np.testing.assert_allclose(F3, F[perm], atol=1e-10)


def test_net_force_and_torque(tiny):
    s = _system()
    _, _, F, W = _ef(tiny, s)
    assert np.abs(F.sum(0)).max() < 1e-10
    np.testing.assert_allclose(W, W.T, atol=1e-10)          # rotation invariance => symmetric virial
    m = molecule_batch(1, seed=8)[0]
    m.species = m.species % 3
    i, j, S = neighbor_list(m.pos, None, m.pbc, 4.0)
    _, _, F, _ = tiny.energy_forces(m.pos, m.species, None, i, j, S)
    assert np.abs(F.sum(0)).max() < 1e-10
    assert np.abs(np.cross(m.pos, F).sum(0)).max() < 1e-9


def test_forces_match_finite_differences(tiny):
    s = _system()
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    E, _, F, _ = tiny.energy_forces(s.pos, s.species, s.cell, i, j, S)
    h = 1e-5
    for k in (0, 7, 23):
        for ax in range(3):
            p = s.pos.copy(); p[k, ax] += h
            Ep = tiny.energy_forces(p, s.species, s.cell, i, j, S)[0]
            p[k, ax] -= 2 * h
            Em = tiny.energy_forces(p, s.species, s.cell, i, j, S)[0]
            fd = -(Ep - Em) / (2 * h)
            assert abs(fd - F[k, ax]) < 1e-7 * max(1.0, np.sqrt((F ** 2).mean()))


def test_virial_matches_strain_derivative(tiny):
    s = _system()
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    _, _, _, W = tiny.energy_forces(s.pos, s.species, s.cell, i, j, S)
    h = 1e-6
    dE = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            E2 = []
            for sg in (1, -1):
                eps = np.zeros((3, 3)); eps[a, b] = sg * h
                M = np.eye(3) + eps
                E2.append(tiny.energy_forces(s.pos @ M.T, s.species, s.cell @ M.T, i, j, S)[0])
            dE[a, b] = (E2[0] - E2[1]) / (2 * h)
    np.testing.assert_allclose(W.T, -dE, atol=1e-6 * max(1.0, np.abs(W).max()))


def test_energy_continuous_across_cutoff(tiny):
    """A pair just inside the cutoff contributes nothing to E and F (envelope and
    bias-free MLPs make every term vanish at r_c), so dropping it is continuous."""
    pos = np.array([[0.0, 0.0, 0.0], [1.1, 0.2, -0.3], [4.0 * (1 - 1e-6), 0.0, 0.0]])
    spec = np.array([0, 1, 2])
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    cross = ((i == 0) & (j == 2)) | ((i == 2) & (j == 0))
    assert cross.sum() == 2
    a = tiny.energy_forces(pos, spec, None, i, j, S)
    b = tiny.energy_forces(pos, spec, None, i[~cross], j[~cross], S[~cross])
    assert abs(a[0] - b[0]) < 1e-12
    np.testing.assert_allclose(a[2], b[2], atol=1e-9)
    # and the crossing pair does matter well inside the cutoff
    pos[2, 0] = 3.0
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    cross = ((i == 0) & (j == 2)) | ((i == 2) & (j == 0))
    a = tiny.energy_forces(pos, spec, None, i, j, S)
    b = tiny.energy_forces(pos, spec, None, i[~cross], j[~cross], S[~cross])
    assert abs(a[0] - b[0]) > 1e-6


def test_pair_potential_when_paths_are_off():
    """theta = 0 removes every many-body term: E of a trimer is the sum of its
    dimer energies (minus the extra shifts)."""
    arch = Arch(n_species=2, lmax=1, n_layers=1, channels=4, two_body=(8,), latent=(8,), edge=(4,))
    w = make_weights(arch, 5)
    w["tp.1"][:] = 0.0
    m = AllegroOracle(arch, w)
    pos = np.array([[0.0, 0.0, 0.0], [1.3, 0.4, 0.0], [0.2, 1.9, 0.7]])
    spec = np.array([0, 1, 1])

    def E(p, sp):
        i, j, S = neighbor_list(p, None, [False] * 3, 4.0)
        return m.energy_forces(p, sp, None, i, j, S)[0]

    mu = w["mu"]
    pair = 0.0
    for a, b in ((0, 1), (0, 2), (1, 2)):
        pair += E(pos[[a, b]], spec[[a, b]]) - mu[spec[a]] - mu[spec[b]]
    assert abs(E(pos, spec) - (pair + mu[spec].sum())) < 1e-12
    w2 = make_weights(arch, 5)          # with paths on, the trimer is not pair-additive
    m2 = AllegroOracle(arch, w2)
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    E3 = m2.energy_forces(pos, spec, None, i, j, S)[0]
    pair2 = 0.0
    for a, b in ((0, 1), (0, 2), (1, 2)):
        ii, jj, SS = neighbor_list(pos[[a, b]], None, [False] * 3, 4.0)
        pair2 += m2.energy_forces(pos[[a, b]], spec[[a, b]], None, ii, jj, SS)[0] - w2["mu"][spec[[a, b]]].sum()
    assert abs(E3 - (pair2 + w2["mu"][spec].sum())) > 1e-6


def test_bilinearity_identity_eq1(tiny):
    """Eq. 1: V^{ij,1} = sum_k w^{ik} (V^{ij,0} x Y^{ik}) path by path (first line)
    equals the oracle's single product with the summed environment (second line)."""
    s = _system(30, seed=6)
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    pos = torch.tensor(s.pos)
    d = tiny.edge_vectors(pos, s.cell, i, j, S)
    feats = {}
    tiny.edge_energies(d, s.species, i, j, s.n_atoms, features=feats)
    Y, V0, w1, V1 = feats["Y"].numpy(), feats["V0"].numpy(), feats["w1"].numpy(), feats["V1"].numpy()
    irs = tiny.irreps
    paths = so3.layer_paths(irs[0], irs[1], 2)
    cnt = {}
    for _, _, o in paths:
        cnt[o] = cnt.get(o, 0) + 1
    theta = make_weights(TINY, 3)["tp.1"]
    nu = 1 / math.sqrt(TINY.avg_num_neighbors)
    for e in (0, 5, 31, len(i) - 1):
        ks = np.nonzero(i == i[e])[0]
        ref = np.zeros((4, 9))
        for k in ks:
            for (l1, p1), l2, (lo, po) in paths:
                th = float(theta[lo, 0 if po == 1 else 1, l1, 0 if p1 == 1 else 1, l2]) / math.sqrt(cnt[(lo, po)])
                C = so3.coupling_tensor(l1, l2, lo)
                yk = nu * w1[k, :, l2][:, None] * Y[k, l2 * l2:(l2 + 1) ** 2][None, :]
                ref[:, lo * lo:(lo + 1) ** 2] += th * np.einsum("abc,ua,ub->uc", C, V0[e][:, l1 * l1:(l1 + 1) ** 2], yk)
        np.testing.assert_allclose(V1[e], ref, atol=1e-12)


def test_dimer_closed_form():
    """One channel, l_max = 0, width-1 MLPs: the energy of a dimer written out by hand."""
    arch = Arch(n_species=1, lmax=0, n_layers=1, channels=1, two_body=(1,), latent=(1,), edge=(),
                n_bessel=1)
    w = make_weights(arch, 0)
    w["two_body.0"][:] = [[0.3, -0.2, 0.9]]
    w["embed"][:] = [[1.7]]
    w["env.1"][:] = [[-0.8]]
    w["tp.1"][:] = 0.0
    w["tp.1"][0, 0, 0, 0, 0] = 1.3
    w["latent.1.0"][:] = [[0.6, 2.0]]
    w["edge.0"][:] = [[1.5]]
    w["sigma"][:] = [1.2]
    w["mu"][:] = [-3.0]
    m = AllegroOracle(arch, w)
    r = 2.3
    pos = np.array([[0.0, 0.0, 0.0], [0.0, r, 0.0]])
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    E, Ea, _, _ = m.energy_forces(pos, np.zeros(2, int), None, i, j, S)
    f32 = lambda v: float(np.float32(v))
    sil = lambda z: z / (1 + math.exp(-z))
    B = math.sqrt(2 / 4.0) * math.sin(math.pi * r / 4.0) / r
    x = r / 4.0
    u = 1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8
    x0 = u * sil(f32(0.3) + f32(-0.2) + f32(0.9) * B)
    V0 = f32(1.7) * x0
    Gam = f32(-0.8) * x0 / math.sqrt(27.0)
    s = f32(1.3) * V0 * Gam
    x1 = u * sil(f32(0.6) * x0 + f32(2.0) * s)
    Eij = f32(1.5) * x1
    assert abs(E - 2 * (1.2 * Eij - 3.0)) < 1e-12
    np.testing.assert_allclose(Ea, [1.2 * Eij - 3.0] * 2, atol=1e-12)


def test_chunked_equals_single_chunk(tiny):
    s = _system(60, seed=1)
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    a = tiny.energy_forces(s.pos, s.species, s.cell, i, j, S, chunk_atoms=7)
    b = tiny.energy_forces(s.pos, s.species, s.cell, i, j, S, chunk_atoms=10_000)
    assert abs(a[0] - b[0]) < 1e-10
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_allclose(x, y, atol=1e-10)


def test_nve_energy_drift_small():
    """Velocity Verlet with the oracle's forces conserves E_kin + E_pot."""
    arch = Arch(n_species=2, lmax=1, n_layers=1, channels=4, two_body=(8,), latent=(8,), edge=(4,))
    m = AllegroOracle(arch, make_weights(arch, 2))
    s = random_box(32, (32 / 0.1) ** (1 / 3), seed=3, species_counts=(21, 11))
    masses = np.array([SPECIES_MASSES[0], SPECIES_MASSES[1]])[s.species]

    def force_fn(p):
        i, j, S = neighbor_list(p, s.cell, s.pbc, 4.0)
        E, _, F, _ = m.energy_forces(p, s.species, s.cell, i, j, S)
        return E, F

    rng = np.random.default_rng(0)
    vel0 = rng.normal(size=(32, 3)) * np.sqrt(0.0257 * 9.648533212e-3 / masses[:, None]) * 0.3
    devs = []
    for dt, n in ((0.25, 200), (0.125, 400)):           # same 50 fs of simulated time
        E0, F = force_fn(s.pos)
        pos, vel = s.pos.copy(), vel0.copy()
        Etot0 = E0 + kinetic_energy(vel, masses)
        dev = 0.0
        for _ in range(n):
            pos, vel, F, E = verlet_step(pos, vel, F, masses, dt, force_fn)
            dev = max(dev, abs(E + kinetic_energy(vel, masses) - Etot0))
        devs.append(dev)
    assert devs[0] / 32 < 1e-4
    # second-order integrator with consistent forces: halving dt cuts the error ~4x
    assert 2.5 < devs[0] / devs[1] < 6.5


def test_c1_runs_and_is_finite():
    s, arch, w = make_config("c1")
    m = AllegroOracle(arch, w)
    E, Ea, F, W = _ef(m, s)
    assert np.isfinite(E) and np.all(np.isfinite(F)) and np.all(np.isfinite(W))
    assert abs(Ea.sum() - E) < 1e-10


# ---------------------------------------------------------------------------
# Heteronuclear closed forms: which atom an edge energy belongs to, and which
# one-hot block carries the centre's species, written out by hand.
# ---------------------------------------------------------------------------
HETERO = Arch(n_species=2, lmax=0, n_layers=1, channels=1, two_body=(2,), latent=(2,), edge=(2,),
              n_bessel=1)


def _hetero_weights():
    """Two species with different sigma and mu, a two-body layer whose centre
    and neighbour one-hot columns differ, a two-wide latent MLP and a linear
    edge MLP with one hidden layer (so E_ij = W_e1 W_e0 x^1)."""
    w = make_weights(HETERO, 0)
    #                      Zi=0   Zi=1   Zj=0   Zj=1   B
    w["two_body.0"][:] = [[0.40, -0.70, 1.10, 0.20, 0.90],
                          [-0.50, 0.30, 0.60, -1.20, 0.45]]
    w["embed"][:] = [[1.7, -0.4]]
    w["env.1"][:] = [[-0.8, 0.55]]
    w["tp.1"][:] = 0.0
    w["tp.1"][0, 0, 0, 0, 0] = 1.3
    w["latent.1.0"][:] = [[0.6, -0.9, 2.0],
                          [0.25, 0.7, -1.5]]
    w["edge.0"][:] = [[1.5, -0.3],
                      [0.2, 0.8]]
    w["edge.1"][:] = [[0.9, -1.1]]
    w["sigma"][:] = [1.2, 0.7]
    w["mu"][:] = [-3.0, 2.5]
    return w


def _hand_energies(pos, spec, w, to_neighbour=False, swap_blocks=False):
    """Per-atom energies of a 1-layer, l_max 0, one-channel model by hand:
    the Allegro sums of Sec. "Allegro" with E_i = sum over the edges whose
    CENTRE is i, the two-body input [onehot(Z_i) | onehot(Z_j) | B(r_ij)],
    Gamma_i = nu sum_{k in N(i)} w^1_ik Y_00 (Y_00 = 1 in the component
    normalisation), V^1_ij = theta V^0_ij Gamma_i, all in plain floats.
    `to_neighbour` / `swap_blocks` make the two plausible mistakes on purpose
    (edge energy given to j; one-hot blocks in the order Z_j, Z_i)."""
    f = lambda a: [[float(np.float32(x)) for x in row] for row in np.atleast_2d(a)]
    W2, We, Wv, Wl, E0, E1 = (f(w[k]) for k in ("two_body.0", "embed", "env.1", "latent.1.0",
                                                  "edge.0", "edge.1"))
    th = float(np.float32(1.3))
    sig, mu = w["sigma"], w["mu"]
    sil = lambda z: z / (1.0 + math.exp(-z))
    rc, nu, n = 4.0, 1.0 / math.sqrt(27.0), len(spec)
    edges = [(a, b) for a in range(n) for b in range(n)
             if a != b and np.linalg.norm(pos[b] - pos[a]) < rc]
    x0, uu = {}, {}
    for a, b in edges:
        r = float(np.linalg.norm(pos[b] - pos[a]))
        B = math.sqrt(2 / rc) * math.sin(math.pi * r / rc) / r
        x = r / rc
        uu[a, b] = 1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8
        zc, zn = (spec[b], spec[a]) if swap_blocks else (spec[a], spec[b])
        inp = [1.0 if zc == 0 else 0.0, 1.0 if zc == 1 else 0.0,
               1.0 if zn == 0 else 0.0, 1.0 if zn == 1 else 0.0, B]
        x0[a, b] = [uu[a, b] * sil(sum(W2[o][k] * inp[k] for k in range(5))) for o in range(2)]
    gam = {a: nu * sum(Wv[0][0] * x0[c, d][0] + Wv[0][1] * x0[c, d][1] for c, d in edges if c == a)
           for a in range(n)}
    Eat = [0.0] * n
    for a, b in edges:
        V0 = We[0][0] * x0[a, b][0] + We[0][1] * x0[a, b][1]
        s = th * V0 * gam[a]
        h = [x0[a, b][0], x0[a, b][1], s]
        x1 = [uu[a, b] * sil(sum(Wl[o][k] * h[k] for k in range(3))) for o in range(2)]
        hid = [E0[o][0] * x1[0] + E0[o][1] * x1[1] for o in range(2)]
        Eat[b if to_neighbour else a] += E1[0][0] * hid[0] + E1[0][1] * hid[1]
    return [sig[spec[a]] * Eat[a] + mu[spec[a]] for a in range(n)]


@pytest.mark.parametrize("case", ["dimer", "trimer"])
def test_heteronuclear_closed_form(case):
    """Per-atom and total energies of a heteronuclear dimer and an asymmetric
    trimer against the hand evaluation.  Swapping centre and neighbour in the
    per-atom sum, or the order of the one-hot blocks, changes every E_i here."""
    w = _hetero_weights()
    m = AllegroOracle(HETERO, w)
    if case == "dimer":
        pos = np.array([[0.0, 0.0, 0.0], [0.4, 2.1, -0.3]])
        spec = np.array([0, 1])
    else:
        pos = np.array([[0.0, 0.0, 0.0], [1.9, 0.3, 0.0], [0.5, 2.6, 0.8]])
        spec = np.array([1, 0, 1])
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    E, Ea, _, _ = m.energy_forces(pos, spec, None, i, j, S)
    ref = _hand_energies(pos, spec, w)
    np.testing.assert_allclose(Ea, ref, rtol=0, atol=1e-12)
    assert abs(E - sum(ref)) < 1e-12
    # the case discriminates: attributing each edge to its neighbour, or
    # exchanging the one-hot blocks, moves every per-atom energy
    for bad in (dict(to_neighbour=True), dict(swap_blocks=True)):
        wrong = _hand_energies(pos, spec, w, **bad)
        assert min(abs(x - y) for x, y in zip(ref, wrong)) > 1e-3, bad
