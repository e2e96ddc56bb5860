"""Velocity-Verlet MD on the GPU (allegro_md_verlet) against the oracle's
Verlet with oracle forces, and energy conservation."""
import numpy as np
import pytest

from gpu_util import lib_model
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from oracle.verlet import verlet_step, kinetic_energy
from synth import make_config, weights_to_blob, lattice_box, ARCHS, make_weights, SPECIES_MASSES

pytestmark = pytest.mark.gpu


def _velocities(n, masses, T_K, seed):
    rng = np.random.default_rng(seed)
    kT = 8.617333e-5 * T_K                       # eV
    return rng.normal(size=(n, 3)) * np.sqrt(kT * 9.648533212e-3 / masses[:, None])


def test_md_matches_oracle_verlet_c1():
    s, arch, w = make_config("c1")
    type_masses = np.array(SPECIES_MASSES[:2])
    masses = type_masses[s.species]
    vel0 = _velocities(s.n_atoms, masses, 300.0, 1)
    m = lib_model(weights_to_blob(arch, w))
    pos = s.pos.copy(); vel = vel0.copy()
    Ep, Ek = m.md_verlet(pos, vel, s.species, type_masses, dt=0.5, n_steps=20, cell=s.cell)
    m.close()
    orc = AllegroOracle(arch, w)

    def force_fn(p):
        i, j, S = neighbor_list(p, s.cell, s.pbc, 4.0)
        E, _, F, _ = orc.energy_forces(p, s.species, s.cell, i, j, S)
        return E, F

    p, v = s.pos.copy(), vel0.copy()
    E0, F = force_fn(p)
    assert abs(Ep[0] - E0) < 1e-5 * abs(E0)
    assert abs(Ek[0] - kinetic_energy(v, masses)) < 1e-12
    for k in range(20):
        p, v, F, E = verlet_step(p, v, F, masses, 0.5, force_fn)
        assert abs(Ep[k + 1] - E) < 1e-5 * max(1.0, abs(E))
    # bounds from the float32 force gate |dF| <= 1e-4 rms|F| accumulated over the run:
    # |dv| <= n dt a_conv |dF| / m_min,  |dx| <= n dt |dv|
    rms = np.sqrt((F ** 2).mean())
    dv = 20 * 0.5 * 9.648533212e-3 * 1e-4 * rms / masses.min()
    np.testing.assert_allclose(vel, v, rtol=0, atol=dv)
    np.testing.assert_allclose(pos, p, rtol=0, atol=20 * 0.5 * dv)
    assert abs(Ek[-1] - kinetic_energy(v, masses)) < 1e-4 * Ek[-1]


def test_md_energy_conservation_fp32():
    arch = ARCHS["c2"]
    w = make_weights(arch, 1)
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=12)
    masses = np.array(SPECIES_MASSES)
    vel = _velocities(s.n_atoms, masses[s.species], 300.0, 2)
    m = lib_model(weights_to_blob(arch, w))
    pos = s.pos.copy()
    Ep, Ek = m.md_verlet(pos, vel, s.species, masses, dt=0.25, n_steps=200, cell=s.cell)
    m.close()
    Et = Ep + Ek
    assert np.all(np.isfinite(Et))
    assert np.abs(Et - Et[0]).max() / s.n_atoms < 1e-4
    assert np.abs(Ek - Ek[0]).max() > 1e-3            # the system actually moves


def test_md_bf16_runs_and_device_buffers():
    import torch
    s, arch, w = make_config("c1")
    type_masses = np.array(SPECIES_MASSES[:2])
    vel0 = _velocities(s.n_atoms, type_masses[s.species], 300.0, 3)
    m = lib_model(weights_to_blob(arch, w), precision="bf16")
    pos = torch.tensor(s.pos, device="cuda"); vel = torch.tensor(vel0, device="cuda")
    Ep, Ek = m.md_verlet(pos, vel, torch.tensor(s.species, dtype=torch.int32, device="cuda"), type_masses,
                         dt=0.5, n_steps=10, cell=s.cell)
    m.close()
    assert np.all(np.isfinite(Ep + Ek)) and torch.isfinite(pos).all()
    assert not torch.equal(pos.cpu(), torch.tensor(s.pos))


# ---------------------------------------------------------------------------
# Verlet skin: the exact list filtered from a candidate list at r_c + skin,
# rebuilt once an atom has moved skin / 2.  The energies must be those of a
# rebuild every step (same pair sets), and the trajectory must follow the
# oracle's rebuild-every-step Verlet run.
# ---------------------------------------------------------------------------
def test_md_skin_matches_rebuild_every_step_and_oracle():
    s, arch, w = make_config("c1")
    type_masses = np.array(SPECIES_MASSES[:2])
    masses = type_masses[s.species]
    vel0 = _velocities(s.n_atoms, masses, 600.0, 5)
    blob = weights_to_blob(arch, w)
    runs = {}
    for skin in (0.0, 0.3):
        m = lib_model(blob)
        m.set_md_skin(skin)
        pos, vel = s.pos.copy(), vel0.copy()
        Ep, Ek = m.md_verlet(pos, vel, s.species, type_masses, dt=0.5, n_steps=40, cell=s.cell)
        runs[skin] = (Ep, Ek, pos, vel, m.md_rebuilds())
        m.close()
    Ep0, Ek0, p0, v0, nb0 = runs[0.0]
    Ep1, Ek1, p1, v1, nb1 = runs[0.3]
    assert nb0 == 41 and 1 <= nb1 < 41, (nb0, nb1)
    # same pair sets every step: only the float32 summation order inside rows differs.  A
    # reordered float32 sum of n terms moves by at most n 2^-24 of their magnitudes, so the
    # forces of the two runs differ by at most (longest row) 2^-24 RMS|F| per step; integrated
    # over the 40 steps like the oracle comparison below, that bounds the position difference.
    np.testing.assert_allclose(Ep1, Ep0, rtol=0, atol=1e-6 * np.abs(Ep0).max())
    orc = AllegroOracle(arch, w)
    i0, _, _ = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    _, _, F0, _ = orc.energy_forces(s.pos, s.species, s.cell, *neighbor_list(s.pos, s.cell, s.pbc, 4.0))
    reorder = np.bincount(i0).max() * 2.0 ** -24
    dv_reorder = 40 * 0.5 * 9.648533212e-3 * reorder * np.sqrt((F0 ** 2).mean()) / masses.min()
    np.testing.assert_allclose(p1, p0, rtol=0, atol=40 * 0.5 * dv_reorder)
    # and the oracle's Verlet with a fresh brute-force-rule list every step

    def force_fn(p):
        i, j, S = neighbor_list(p, s.cell, s.pbc, 4.0)
        E, _, F, _ = orc.energy_forces(p, s.species, s.cell, i, j, S)
        return E, F

    p, v = s.pos.copy(), vel0.copy()
    _, F = force_fn(p)
    for k in range(40):
        p, v, F, E = verlet_step(p, v, F, masses, 0.5, force_fn)
        assert abs(Ep1[k + 1] - E) < 1e-5 * max(1.0, abs(E))
    rms = np.sqrt((F ** 2).mean())
    dv = 40 * 0.5 * 9.648533212e-3 * 1e-4 * rms / masses.min()
    np.testing.assert_allclose(v1, v, rtol=0, atol=dv)
    np.testing.assert_allclose(p1, p, rtol=0, atol=40 * 0.5 * dv)


def test_md_skin_energy_conservation_and_lists():
    """NVE with the skin on a 1,000-atom box (2 layers, l_max 2), and the list
    left in the context after the run equals the oracle's list of the final
    positions."""
    arch = ARCHS["c2"]
    w = make_weights(arch, 1)
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=12)
    masses = np.array(SPECIES_MASSES)
    vel = _velocities(s.n_atoms, masses[s.species], 300.0, 2)
    m = lib_model(weights_to_blob(arch, w))
    m.set_md_skin(0.5)
    pos = s.pos.copy()
    Ep, Ek = m.md_verlet(pos, vel, s.species, masses, dt=0.25, n_steps=200, cell=s.cell)
    nb = m.md_rebuilds()
    from gpu_util import assert_same_edges
    assert_same_edges(m.get_neighbors(), neighbor_list(pos, s.cell, s.pbc, 4.0))
    m.close()
    Et = Ep + Ek
    assert np.all(np.isfinite(Et))
    assert np.abs(Et - Et[0]).max() / s.n_atoms < 1e-4
    assert nb < 100, nb                                # the candidate list is reused


def test_md_skin_rejects_bad_values():
    from paper_2304_10061_gb300 import AllegroError
    s, arch, w = make_config("c1")
    m = lib_model(weights_to_blob(arch, w))
    for bad in (-0.1, float("nan"), float("inf"), 100.0):
        with pytest.raises(AllegroError):
            m.set_md_skin(bad)
    m.set_md_skin(0.0)
    m.close()
