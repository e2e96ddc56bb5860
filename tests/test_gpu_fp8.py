"""FP8 precision (E4M3 MLP GEMMs on tcgen05 kind::f8f6f4, per-tensor scales)
against the FP64 oracle, through the C ABI.

Gates, from the arithmetic: E4M3 keeps 3 mantissa bits (unit roundoff 2^-4),
bfloat16 keeps 7 (2^-8), so every error of the BF16 path's gates is scaled by
16: force RMS error < 32 % of RMS|F|, max < 3.2 RMS|F|, per-atom energy < 0.16
of max(|E_i|, rms E_i), virial < 0.8 of max|W|.  These only say the path is
not broken; the pin is the comparison with the oracle under the same E4M3
rounding of every MLP product (tests/fp8_util.py): the library's force error
must be within a factor 2 of the error that rounding predicts, both ways (much
smaller would mean the products are not in E4M3, much larger a wrong scale,
layout or format).
"""
import numpy as np
import pytest

from fp8_util import E4MOracle
from gpu_util import BF16_F_RMS, errors, lib_model, assert_same_edges
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from synth import Arch, ARCHS, make_weights, weights_to_blob, lattice_box, make_config

pytestmark = pytest.mark.gpu

FP8_F_RMS = 16 * BF16_F_RMS
FP8_F_MAX = 16 * 10 * BF16_F_RMS
FP8_E = 16 * 1e-2
FP8_W = 16 * 5e-2

L3X3 = Arch(n_species=2, lmax=3, n_layers=3, channels=16, two_body=(32,), latent=(64,), edge=(8,))
L1X2 = Arch(n_species=2, lmax=1, n_layers=2, channels=32, two_body=(64,), latent=(64, 96), edge=(16, 8))
L3X3C128 = Arch(n_species=2, lmax=3, n_layers=3, channels=128, two_body=(64,), latent=(64,), edge=(16,))


def _cases():
    s1, a1, w1 = make_config("c1")
    s2 = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=5)
    s3 = lattice_box(200, (200 / 0.1) ** (1 / 3), seed=12)
    s3.species = s3.species % 2
    sl = lattice_box(500, (500 / 0.1) ** (1 / 3), seed=8)
    sl.species = sl.species % 2
    s3c = lattice_box(120, (120 / 0.1) ** (1 / 3), seed=14)
    s3c.species = s3c.species % 2
    return {
        "c1": (a1, w1, s1),
        "c2arch_1000": (ARCHS["c2"], make_weights(ARCHS["c2"], 1), s2),
        "three_layers_lmax3": (L3X3, make_weights(L3X3, 10), s3),
        "lmax1_two_layers": (L1X2, make_weights(L1X2, 6), sl),
        "three_layers_lmax3_C128": (L3X3C128, make_weights(L3X3C128, 13), s3c),
    }


CASES = _cases()
_REF = {}


def _reference(name):
    """(edges, exact oracle result, oracle result under E4M3 rounding of the MLP products)"""
    if name not in _REF:
        arch, w, s = CASES[name]
        i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c)
        exact = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S)
        rounded = E4MOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S)
        _REF[name] = ((i, j, S), exact, rounded)
    return _REF[name]


def _run(arch, w, s, prec, chunk=0):
    m = lib_model(weights_to_blob(arch, w), precision=prec)
    if chunk:
        m.reserve(0, 0, 0, chunk)
    m.neighbors(s.pos, s.species, s.cell)
    out = m.energy_forces()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    edges = m.get_neighbors()
    m.close()
    return res, edges


@pytest.mark.parametrize("name", list(CASES))
def test_fp8_matches_oracle(name):
    arch, w, s = CASES[name]
    res, edges = _run(arch, w, s, "fp8")
    eo, (E0, Ea0, F0, W0), (E8, Ea8, F8, W8) = _reference(name)
    assert_same_edges(edges, eo)
    err = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)
    pred = errors(Ea8, F8, W8, Ea0, F0, W0)
    print(name, "library", err, "E4M3-rounded oracle", pred)
    assert np.all(np.isfinite(res["F"])) and np.isfinite(res["E"][0])
    assert err["f_rms"] < FP8_F_RMS, err
    assert err["f_max"] < FP8_F_MAX, err
    assert err["e_rel"] < FP8_E, err
    assert err["w_rel"] < FP8_W, err
    assert 0.5 * pred["f_rms"] < err["f_rms"] < 2.0 * pred["f_rms"], (err, pred)


def test_fp8_error_above_bf16():
    """E4M3 products are coarser than bfloat16 ones: the FP8 force error is several times the BF16 one."""
    arch, w, s = CASES["c2arch_1000"]
    _, (E0, Ea0, F0, W0), _ = _reference("c2arch_1000")
    e = {}
    for prec in ("bf16", "fp8"):
        res, _ = _run(arch, w, s, prec)
        e[prec] = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)["f_rms"]
    assert e["fp8"] > 4 * e["bf16"], e


def test_fp8_deterministic():
    arch, w, s = CASES["c2arch_1000"]
    a, _ = _run(arch, w, s, "fp8")
    b, _ = _run(arch, w, s, "fp8")
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_fp8_chunked_within_gate():
    """Chunks of whole rows: each chunk's activations get their own per-tensor scales,
    so the result differs from the single pass at the level of the E4M3 rounding only."""
    arch, w, s = CASES["c2arch_1000"]
    _, (E0, Ea0, F0, W0), (E8, Ea8, F8, W8) = _reference("c2arch_1000")
    res, _ = _run(arch, w, s, "fp8", chunk=4000)
    err = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)
    pred = errors(Ea8, F8, W8, Ea0, F0, W0)
    assert err["f_rms"] < 2.0 * pred["f_rms"], (err, pred)


def test_fp8_degenerate_systems():
    """Empty input, one atom without neighbours, isolated atoms beside a bonded pair."""
    import torch
    arch, w, _ = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w), precision="fp8")
    m.neighbors(np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 10)
    out = m.energy_forces()
    assert out["E"].item() == 0.0 and out["F"].numel() == 0
    m.neighbors(np.array([[1.0, 2.0, 3.0]]), np.array([1], np.int32), np.eye(3) * 20)
    out = m.energy_forces()
    assert out["E"].item() == pytest.approx(w["mu"][1], abs=1e-12)
    assert torch.all(out["F"] == 0)
    pos = np.array([[0.0, 0, 0], [1.5, 0, 0], [20, 0, 0], [0, 20, 0]])
    m.neighbors(pos, np.array([0, 1, 1, 0], np.int32), None)
    out = m.energy_forces()
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    E0, Ea0, F0, W0 = AllegroOracle(arch, w).energy_forces(pos, [0, 1, 1, 0], None, i, j, S)
    err = errors(out["E_atom"].cpu().numpy(), out["F"].cpu().numpy(), None, Ea0, F0, W0)
    assert err["e_rel"] < FP8_E and err["f_max"] < FP8_F_MAX, err
    m.close()


def test_fp8_batched_molecules_per_structure():
    """Packed uneven molecules: per-molecule energies and forces within the FP8 gates."""
    from synth import molecule_batch
    from synth.structures import pack
    arch, w = ARCHS["c2"], make_weights(ARCHS["c2"], 1)
    mols = molecule_batch(48, seed=2)
    pos, spec, offs = pack(mols)
    m = lib_model(weights_to_blob(arch, w), precision="fp8")
    m.neighbors_batched(offs, pos, spec)
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    m.close()
    orc = AllegroOracle(arch, w)
    for b in (0, 17, 47):
        mb = mols[b]
        i, j, S = neighbor_list(mb.pos, None, mb.pbc, 4.0)
        E0, Ea0, F0, W0 = orc.energy_forces(mb.pos, mb.species, None, i, j, S)
        sl = slice(offs[b], offs[b + 1])
        err = errors(out["E_atom"][sl], out["F"][sl], out["virial"][b], Ea0, F0, W0)
        assert err["f_rms"] < FP8_F_RMS and err["e_rel"] < FP8_E, (b, err)


def test_fp8_graph_replay_equals_eager():
    """The amax slots are cleared inside the captured work: replays equal eager launches bitwise."""
    arch, w, s = CASES["c2arch_1000"]
    blob = weights_to_blob(arch, w)
    eager = lib_model(blob, precision="fp8")
    eager.neighbors(s.pos, s.species, s.cell)
    ref = {k: v.cpu().numpy() for k, v in eager.energy_forces().items()}
    g = lib_model(blob, precision="fp8")
    g.set_graphs(True)
    g.neighbors(s.pos, s.species, s.cell)
    for _ in range(4):
        o = {k: v.cpu().numpy() for k, v in g.energy_forces().items()}
        for k in ref:
            np.testing.assert_array_equal(o[k], ref[k])
    assert g.autotune_report()["graph_replays"] >= 2
    eager.close()
    g.close()


def test_fp8_pair_cutoffs_and_zbl():
    """The per-pair cutoff table and the ZBL term (float32 arithmetic outside the GEMMs) on the FP8 path."""
    from dataclasses import replace
    from synth import SPECIES_Z, paper_pair_cutoffs
    arch = replace(Arch(n_species=5, lmax=2, n_layers=2, channels=16, two_body=(32,), latent=(32,), edge=(8,),
                        zbl_z=SPECIES_Z), pair_rc=paper_pair_cutoffs())
    w = make_weights(arch, 23)
    s = lattice_box(800, (800 / 0.1) ** (1 / 3), seed=42)
    m = lib_model(weights_to_blob(arch, w), precision="fp8")
    m.set_pair_cutoffs(np.asarray(arch.pair_rc))
    m.set_zbl(SPECIES_Z)
    m.neighbors(s.pos, s.species, s.cell)
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    m.close()
    ed = neighbor_list(s.pos, s.cell, s.pbc, 4.0, species=s.species, pair_rc=arch.pair_rc)
    E0, Ea0, F0, W0 = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, *ed)
    err = errors(out["E_atom"], out["F"], out["virial"][0], Ea0, F0, W0)
    assert err["f_rms"] < FP8_F_RMS and err["e_rel"] < FP8_E and err["w_rel"] < FP8_W, err


def test_fp8_md_and_autotune():
    """Velocity-Verlet steps on the FP8 path stay finite and move the atoms; the autotuner's
    configuration (its chunk sizes give each chunk its own activation scales) stays within the
    gates."""
    from synth import SPECIES_MASSES
    arch, w, s = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w), precision="fp8")
    type_masses = np.array(SPECIES_MASSES[:2])
    rng = np.random.default_rng(3)
    vel = rng.normal(size=(s.n_atoms, 3)) * np.sqrt(0.0257 * 9.648533212e-3 / type_masses[s.species][:, None])
    pos = s.pos.copy()
    Ep, Ek = m.md_verlet(pos, vel, s.species, type_masses, dt=0.5, n_steps=10, cell=s.cell)
    m.close()
    assert np.all(np.isfinite(Ep + Ek)) and np.all(np.isfinite(pos))
    assert not np.array_equal(pos, s.pos)
    arch, w, s = CASES["c2arch_1000"]
    _, (E0, Ea0, F0, W0), (E8, Ea8, F8, W8) = _reference("c2arch_1000")
    m = lib_model(weights_to_blob(arch, w), precision="fp8")
    m.set_autotune(True)
    m.neighbors(s.pos, s.species, s.cell)
    for _ in range(2):
        out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    m.close()
    err = errors(out["E_atom"], out["F"], out["virial"][0], Ea0, F0, W0)
    pred = errors(Ea8, F8, W8, Ea0, F0, W0)
    assert err["f_rms"] < 2.0 * pred["f_rms"] and err["e_rel"] < FP8_E, (err, pred)
