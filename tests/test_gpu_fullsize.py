"""Full-size workloads on the GPU, checked on sampled outputs the oracle computes
one by one (strict locality: E_i needs only atom i's row; F_k needs the rows of
k and of every atom that has k as a neighbour).

  23,552-atom box (2 layers, l_max 2, 64 channels)   float32 and BF16
  1,048,576-atom box (same model, the benchmarked workload)   float32 and BF16
"""
import numpy as np
import pytest

from gpu_util import BF16_F_RMS, FP32_E, FP32_F, lib_model
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from synth import make_config, weights_to_blob

pytestmark = pytest.mark.gpu


def _sampled_check(name, prec, n_e=48, n_f=12):
    s, arch, w = make_config(name)
    m = lib_model(weights_to_blob(arch, w), precision=prec)
    m.neighbors(s.pos, s.species, s.cell)
    out = m.energy_forces()
    Ea = out["E_atom"].cpu().numpy()
    F = out["F"].cpu().numpy()
    W = out["virial"].cpu().numpy()[0]
    gi, gj, _ = m.get_neighbors()
    m.close()
    rng = np.random.default_rng(11)
    orc = AllegroOracle(arch, w)
    # energies of sampled centres
    ce = np.sort(rng.choice(s.n_atoms, n_e, replace=False))
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c, centers=ce)
    _, Ea0, _, _ = orc.energy_forces(s.pos, s.species, s.cell, i, j, S, centers=ce)
    scale = np.sqrt((Ea ** 2).mean())
    e_err = np.abs(Ea[ce] - Ea0[ce]) / np.maximum(np.abs(Ea0[ce]), scale)
    # forces on sampled atoms: all rows that contain k, plus k's own row
    fk = np.sort(rng.choice(s.n_atoms, n_f, replace=False))
    rows = np.unique(np.concatenate([fk, gi[np.isin(gj, fk)]]))
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c, centers=rows)
    _, _, F0, _ = orc.energy_forces(s.pos, s.species, s.cell, i, j, S, centers=rows)
    rms = np.sqrt((F ** 2).mean())
    dF = F[fk] - F0[fk]
    # whole-system invariants that hold at any size
    net = np.abs(F.sum(0)).max() / rms
    return e_err, dF, rms, net, W


@pytest.mark.parametrize("name", ["c2", "c4"])
def test_fullsize_fp32(name):
    e_err, dF, rms, net, W = _sampled_check(name, "fp32")
    assert e_err.max() < FP32_E, e_err.max()
    assert np.abs(dF).max() < FP32_F * rms, np.abs(dF).max() / rms
    assert net < 1e-6
    assert np.abs(W - W.T).max() < 1e-6 * np.abs(W).max()


@pytest.mark.parametrize("name", ["c2", "c4"])
def test_fullsize_bf16(name):
    e_err, dF, rms, net, W = _sampled_check(name, "bf16")
    assert np.sqrt((dF ** 2).mean()) < BF16_F_RMS * rms
    assert e_err.max() < 1e-2
    assert net < 1e-4
