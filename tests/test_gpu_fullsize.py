"""Full-size workloads on the GPU, checked on sampled outputs the oracle computes
one by one (strict locality: E_i needs only atom i's row; F_k needs the rows of
k and of every atom that has k as a neighbour).

  23,552-atom box (2 layers, l_max 2, 64 channels)   float32 and BF16
  1,048,576-atom box (same model, the benchmarked workload)   float32 and BF16,
      TF32 (the paper's production setting), and BF16 under the paper's
      per-ordered-species-pair cutoff table
  4,194,304-atom box (3 layers, l_max 3, 128 channels)   BF16, as benchmarked
  2048 packed gas-phase molecules (2 layers, l_max 2, 64 channels)   float32 and
      BF16 with the autotuner and CUDA-graph replay on, as benchmarked; sampled
      molecules checked whole (they are independent structures)
"""
import numpy as np
import pytest

from gpu_util import BF16_F_RMS, FP32_E, FP32_F, FP32_W, errors, lib_model
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from dataclasses import replace

from synth import make_config, paper_pair_cutoffs, weights_to_blob
from synth.structures import pack

pytestmark = pytest.mark.gpu


def _sampled_check(name, prec, n_e=48, n_f=12, pair_rc=None):
    s, arch, w = make_config(name)
    m = lib_model(weights_to_blob(arch, w), precision=prec)
    if pair_rc is not None:
        m.set_pair_cutoffs(np.asarray(pair_rc))
        arch = replace(arch, pair_rc=pair_rc)
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
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c, centers=ce, species=s.species, pair_rc=pair_rc)
    _, Ea0, _, _ = orc.energy_forces(s.pos, s.species, s.cell, i, j, S, centers=ce)
    scale = np.sqrt((Ea ** 2).mean())
    e_err = np.abs(Ea[ce] - Ea0[ce]) / np.maximum(np.abs(Ea0[ce]), scale)
    # forces on sampled atoms: all rows that contain k, plus k's own row
    fk = np.sort(rng.choice(s.n_atoms, n_f, replace=False))
    rows = np.unique(np.concatenate([fk, gi[np.isin(gj, fk)]]))
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c, centers=rows, species=s.species, pair_rc=pair_rc)
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


def test_fullsize_c4_tf32():
    """The 1M-atom box on the TF32 path (float32 storage, tcgen05 kind::tf32 GEMMs), gated
    like the other reduced-precision GEMM path."""
    e_err, dF, rms, net, W = _sampled_check("c4", "tf32")
    assert np.sqrt((dF ** 2).mean()) < BF16_F_RMS * rms
    assert e_err.max() < 1e-2
    assert net < 1e-4


def test_fullsize_c4_pair_cutoffs_bf16():
    """The 1M-atom box under the paper's per-ordered-species-pair cutoff table, BF16 path:
    the oracle's rows use the same table."""
    e_err, dF, rms, net, W = _sampled_check("c4", "bf16", pair_rc=paper_pair_cutoffs(default=4.0))
    assert np.sqrt((dF ** 2).mean()) < BF16_F_RMS * rms
    assert e_err.max() < 1e-2
    assert net < 1e-4


def test_fullsize_c5_bf16():
    """The 4,194,304-atom three-layer l_max 3 model in the benchmarked precision:
    sampled centres' energies and sampled atoms' forces against the oracle (one
    oracle pass over the union of the rows they need)."""
    s, arch, w = make_config("c5")
    m = lib_model(weights_to_blob(arch, w), precision="bf16")
    m.neighbors(s.pos, s.species, s.cell)
    out = m.energy_forces()
    Ea = out["E_atom"].cpu().numpy()
    F = out["F"].cpu().numpy()
    gi, gj, _ = m.get_neighbors()
    m.close()
    rng = np.random.default_rng(12)
    ce = np.sort(rng.choice(s.n_atoms, 24, replace=False))
    fk = np.sort(rng.choice(s.n_atoms, 6, replace=False))
    # every row that contains a sampled atom k, k's own row, and the sampled centres
    rows = np.unique(np.concatenate([ce, fk, gi[np.isin(gj, fk)]]))
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c, centers=rows)
    _, Ea0, F0, _ = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S, centers=rows)
    scale = np.sqrt((Ea ** 2).mean())
    e_err = np.abs(Ea[ce] - Ea0[ce]) / np.maximum(np.abs(Ea0[ce]), scale)
    rms = np.sqrt((F ** 2).mean())
    dF = F[fk] - F0[fk]
    assert e_err.max() < 1e-2, e_err.max()
    assert np.sqrt((dF ** 2).mean()) < BF16_F_RMS * rms, np.sqrt((dF ** 2).mean()) / rms
    assert np.abs(F.sum(0)).max() / rms < 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fullsize_c3_autotuned_graphs(prec):
    """2048 uneven molecules in one packed list with the autotuner and CUDA-graph
    replay on (tune, capture, replay): the replayed evaluation's per-molecule E,
    F and virial of sampled molecules against the oracle."""
    mols, arch, w = make_config("c3")
    pos, spec, offs = pack(mols)
    m = lib_model(weights_to_blob(arch, w), precision=prec)
    m.set_autotune(True)
    m.set_graphs(True)
    m.neighbors_batched(offs, pos, spec)
    for _ in range(3):
        out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    rep = m.autotune_report()
    m.close()
    assert rep["graph_replays"] >= 1 and len(rep["buckets"]) == 1, rep
    orc = AllegroOracle(arch, w)
    for b in (0, 511, 1024, 1500, 2047):
        mb = mols[b]
        i, j, S = neighbor_list(mb.pos, None, mb.pbc, arch.r_c)
        E0, Ea0, F0, W0 = orc.energy_forces(mb.pos, mb.species, None, i, j, S)
        sl = slice(offs[b], offs[b + 1])
        err = errors(out["E_atom"][sl], out["F"][sl], out["virial"][b], Ea0, F0, W0)
        if prec == "fp32":
            assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F and err["w_rel"] < FP32_W, (b, err)
            assert abs(out["E"][b] - E0) < FP32_E * np.abs(Ea0).sum()
        else:
            assert err["f_rms"] < BF16_F_RMS, (b, err)
