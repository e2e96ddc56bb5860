"""Emulated spatial decomposition on one GPU (the multi-GPU design of Sec.
"Optimized LAMMPS-Kokkos implementation", strict locality): the box split
into 2-8 slabs, each slab's ghost halo gathered device-to-device into its own
buffer (positions on the GPU, index gathers and image shifts on the GPU),
each sub-domain evaluated through allegro_neighbors_local (local atoms the
only centres), ghost forces added back to the atoms they copy.  The summed
energy, forces and virial equal the single-domain evaluation's: the edge sets
and the float64 sums are the same; only the float32 environment sums inside
a row run in another order (the sub-domain's cell grid differs), so the
bound is float32 rounding, well inside the float32 gates."""
import numpy as np
import pytest

from decomp_util import slabs
from gpu_util import lib_model
from synth import ARCHS, lattice_box, make_weights, weights_to_blob

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("P", [2, 4, 8])
def test_emulated_decomposition_equals_single_domain(P, prec):
    import torch
    arch = ARCHS["c2"]
    s = lattice_box(6000, (6000 / 0.1) ** (1 / 3), seed=61)
    m = lib_model(weights_to_blob(arch, make_weights(arch, 1)), precision=prec)
    dev = "cuda"
    pos = torch.tensor(s.pos, device=dev)
    spec = torch.tensor(s.species, dtype=torch.int32, device=dev)
    cell = torch.tensor(s.cell, device=dev)
    n_ref = m.neighbors(pos, spec, cell)
    ref = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    axis = P % 3
    pbc = np.ones(3, np.uint8)
    pbc[axis] = 0
    inv = torch.linalg.inv(cell)
    wrap = torch.floor((pos @ inv)[:, axis])
    E, F, W = 0.0, torch.zeros_like(pos), np.zeros((3, 3))
    n_edges = 0
    for local, ghost, gshift in slabs(s.pos, s.cell, P, arch.r_c, axis):
        li = torch.tensor(local, device=dev)
        gi = torch.tensor(ghost, device=dev)
        gs = torch.tensor(gshift, device=dev, dtype=torch.float64)
        # device-to-device halo exchange: gather, wrap along the axis, apply the image shift
        lp = pos.index_select(0, li) - wrap.index_select(0, li)[:, None] * cell[axis]
        gp = pos.index_select(0, gi) + (gs - wrap.index_select(0, gi))[:, None] * cell[axis]
        sub_pos = torch.cat([lp, gp]).contiguous()
        sub_spec = torch.cat([spec.index_select(0, li), spec.index_select(0, gi)]).contiguous()
        n_edges += m.neighbors_local(len(local), sub_pos, sub_spec, cell, pbc)
        out = m.energy_forces()
        E += out["E"].item()
        W += out["virial"][0].cpu().numpy()
        F.index_add_(0, li, out["F"][:len(local)])
        F.index_add_(0, gi, out["F"][len(local):])
        if len(ghost):
            assert float(out["E_atom"][len(local):].abs().max()) == 0.0     # ghosts carry no energy
    m.close()
    F = F.cpu().numpy()
    assert n_edges == n_ref                            # every edge has exactly one owning sub-domain
    rms = np.sqrt((ref["F"] ** 2).mean())
    tol = 2e-6 if prec == "fp32" else 2e-3        # float32 rounding order / bf16 activations
    assert abs(E - ref["E"][0]) < tol * abs(ref["E"][0])
    assert np.abs(F - ref["F"]).max() < tol * 10 * rms
    assert np.abs(W - ref["virial"][0]).max() < tol * 10 * np.abs(ref["virial"][0]).max()
