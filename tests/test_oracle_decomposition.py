"""Strict locality (Sec. "Optimized LAMMPS-Kokkos implementation": each
sub-domain needs only a ghost halo of width r_c): the FP64 oracle evaluated
slab by slab -- local atoms as the only centres, ghosts as neighbours, ghost
forces added back to the atoms they copy -- reproduces the single-domain
energy, forces and virial to float64 round-off (no GPU).  Pins the
decomposition harness that the GPU test runs through the library."""
import numpy as np
import pytest

from decomp_util import slabs, subdomain_positions
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from synth import Arch, lattice_box, make_weights

ARCH = Arch(n_species=3, lmax=2, n_layers=2, channels=4, two_body=(16,), latent=(16,), edge=(8,))


@pytest.mark.parametrize("P,axis", [(2, 0), (3, 1), (5, 2)])
def test_slab_decomposition_equals_single_domain(P, axis):
    s = lattice_box(300, (300 / 0.1) ** (1 / 3), seed=17)
    s.species = s.species % 3
    m = AllegroOracle(ARCH, make_weights(ARCH, 6))
    E0, Ea0, F0, W0 = m.energy_forces(s.pos, s.species, s.cell, *neighbor_list(s.pos, s.cell, s.pbc, 4.0))
    parts = slabs(s.pos, s.cell, P, 4.0, axis)
    seen = np.concatenate([p[0] for p in parts])
    assert np.array_equal(np.sort(seen), np.arange(s.n_atoms))           # the slabs partition the atoms
    pbc = [True] * 3
    pbc[axis] = False
    E, F, W = 0.0, np.zeros_like(F0), np.zeros((3, 3))
    for part in parts:
        local, ghost, _ = part
        sp, _ = subdomain_positions(s.pos, s.cell, part, axis)
        spec = np.concatenate([s.species[local], s.species[ghost]])
        i, j, S = neighbor_list(sp, s.cell, pbc, 4.0, centers=np.arange(local.size))
        Ek, Eak, Fk, Wk = m.energy_forces(sp, spec, s.cell, i, j, S, centers=np.arange(local.size))
        E += Ek
        np.add.at(F, local, Fk[:local.size])
        np.add.at(F, ghost, Fk[local.size:])
        W += Wk
        np.testing.assert_allclose(Eak[:local.size], Ea0[local], rtol=0, atol=1e-10)
    assert abs(E - E0) < 1e-10 * abs(E0)
    np.testing.assert_allclose(F, F0, rtol=0, atol=1e-10)
    np.testing.assert_allclose(W, W0, rtol=0, atol=1e-9)
