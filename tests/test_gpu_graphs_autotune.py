"""Batching support around the evaluation: CUDA-graph replay and the launch-
configuration autotuner (the fluctuating shapes of Sec. "Optimized
LAMMPS-Kokkos implementation").  Replayed graphs give the eager results
bitwise and follow new positions; a changed edge count falls back to eager
launches; the autotuner's chosen configuration gives the model's results
(against the FP64 oracle, float32 and BF16 gates) for single boxes and
packed molecules, and records its trials."""
import numpy as np
import pytest

from gpu_util import BF16_F_RMS, FP32_E, FP32_F, errors, lib_model
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list, neighbor_list_batched
from synth import ARCHS, lattice_box, make_config, make_weights, molecule_batch, weights_to_blob
from synth.structures import pack

pytestmark = pytest.mark.gpu


def _out(m):
    return {k: v.cpu().numpy() for k, v in m.energy_forces().items()}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_graph_replay_equals_eager(prec):
    arch = ARCHS["c2"]
    blob = weights_to_blob(arch, make_weights(arch, 1))
    s = lattice_box(2000, (2000 / 0.1) ** (1 / 3), seed=51)
    eager = lib_model(blob, precision=prec)
    eager.neighbors(s.pos, s.species, s.cell)
    ref = _out(eager)
    g = lib_model(blob, precision=prec)
    g.set_graphs(True)
    n0 = g.neighbors(s.pos, s.species, s.cell)
    outs = [_out(g) for _ in range(4)]               # eager, capture, replay, replay
    rep = g.autotune_report()
    assert rep["graph_replays"] >= 2 and rep["graph_kernels"] > 10, rep
    for o in outs:
        for k in ref:
            np.testing.assert_array_equal(o[k], ref[k])
    # new positions with the same edges: the replay reads the rebuilt list and gives the new results
    p2 = s.pos + np.random.default_rng(0).normal(scale=1e-7, size=s.pos.shape)
    eager.neighbors(p2, s.species, s.cell)
    ne = g.neighbors(p2, s.species, s.cell)
    ref2 = _out(eager)
    o2 = _out(g)
    for k in ref2:
        np.testing.assert_array_equal(o2[k], ref2[k])
    assert not np.array_equal(o2["F"], ref["F"])
    assert ne == eager.n_edges
    if ne == n0:                                     # same shape: served by the captured graph
        assert g.autotune_report()["graph_replays"] > rep["graph_replays"]
    # a different system: eager fallback, still right
    s3 = lattice_box(1500, (1500 / 0.1) ** (1 / 3), seed=52)
    eager.neighbors(s3.pos, s3.species, s3.cell)
    g.neighbors(s3.pos, s3.species, s3.cell)
    ref3, o3 = _out(eager), _out(g)
    for k in ref3:
        np.testing.assert_array_equal(o3[k], ref3[k])
    eager.close()
    g.close()


def test_graph_replay_batched_molecules():
    mols = molecule_batch(256, seed=53)
    pos, spec, offs = pack(mols)
    arch = ARCHS["c2"]
    blob = weights_to_blob(arch, make_weights(arch, 1))
    eager = lib_model(blob, precision="bf16")
    eager.neighbors_batched(offs, pos, spec)
    ref = _out(eager)
    g = lib_model(blob, precision="bf16")
    g.set_graphs(True)
    g.neighbors_batched(offs, pos, spec)
    for _ in range(3):
        o = _out(g)
    for k in ref:
        np.testing.assert_array_equal(o[k], ref[k])
    assert g.autotune_report()["graph_replays"] >= 1
    eager.close()
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_autotuned_configuration_matches_oracle(prec):
    s, arch, w = make_config("c4sub")
    m = lib_model(weights_to_blob(arch, w), precision=prec)
    m.set_autotune(True)
    m.set_graphs(True)
    m.neighbors(s.pos, s.species, s.cell)
    o = _out(m)
    o = _out(m)                                        # tuned configuration, possibly replayed
    rep = m.autotune_report()
    m.close()
    assert len(rep["buckets"]) == 1
    (bucket,) = rep["buckets"].values()
    assert len(bucket["trials"]) >= (10 if prec == "bf16" else 2), bucket
    best = min(bucket["trials"].values())
    assert best <= list(bucket["trials"].values())[0] + 1e-9
    i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c)
    E0, Ea0, F0, W0 = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S)
    err = errors(o["E_atom"], o["F"], o["virial"][0], Ea0, F0, W0)
    if prec == "fp32":
        assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F, err
    else:
        assert err["f_rms"] < BF16_F_RMS, err


def test_autotune_batched_and_disable():
    mols = molecule_batch(128, seed=54)
    pos, spec, offs = pack(mols)
    arch = ARCHS["c2"]
    w = make_weights(arch, 1)
    m = lib_model(weights_to_blob(arch, w), precision="fp32")
    m.set_autotune(True)
    m.neighbors_batched(offs, pos, spec)
    o = _out(m)
    assert any(k.endswith("batched") for k in m.autotune_report()["buckets"])
    orc = AllegroOracle(arch, w)
    for k, x in enumerate(mols[:8]):
        E0, Ea0, F0, W0 = orc.energy_forces(x.pos, x.species, None, *neighbor_list(x.pos, None, x.pbc, 4.0))
        sl = slice(offs[k], offs[k + 1])
        err = errors(o["E_atom"][sl], o["F"][sl], o["virial"][k], Ea0, F0, W0)
        assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F, (k, err)
    m.set_autotune(False)
    assert m.autotune_report()["current"].startswith("chunk=0,")
    m.close()
