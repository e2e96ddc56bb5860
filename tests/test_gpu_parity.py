"""GPU energies, forces and virial vs the FP64 oracle (through the C ABI).

FP32 path: per-atom energy within 1e-5 of max(|E_i|, rms E_i), max |dF| within
1e-4 rms|F|, virial within 1e-5 of max|W|.  BF16 MLP path: force RMS error
within 2 % of rms|F|, with loose bounds on energies (per-atom energies within 1e-2 of
max(|E_i|, rms E_i): bf16 rounding of the latents, about 2^-9 per element, summed over
a few hundred products per edge and ~25 edges per atom) and on the virial.
"""
import numpy as np
import pytest
import torch

from gpu_util import BF16_F_RMS, FP32_E, FP32_F, FP32_W, errors, lib_model, assert_same_edges
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list, neighbor_list_batched
from synth import Arch, ARCHS, make_weights, weights_to_blob, lattice_box, random_box, molecule_batch, make_config
from synth.structures import pack

pytestmark = pytest.mark.gpu

TINY2 = Arch(n_species=3, lmax=2, n_layers=2, channels=8, two_body=(16, 32), latent=(32, 32), edge=(8,))
TINY1 = Arch(n_species=3, lmax=2, n_layers=1, channels=16, two_body=(24,), latent=(40,), edge=())
L1X2 = Arch(n_species=2, lmax=1, n_layers=2, channels=32, two_body=(64,), latent=(64, 96), edge=(16, 8))
# 128 channels: four channels per lane in the row kernels
C128 = Arch(n_species=2, lmax=2, n_layers=2, channels=128, two_body=(64, 128), latent=(128,), edge=())
# dense rows (~85 neighbours): rows longer than one staged segment of the row kernels
DENSE = Arch(n_species=3, lmax=2, n_layers=2, channels=16, two_body=(32,), latent=(32,), edge=())
# 1024-wide MLPs (the paper's production widths): the BF16 path's heads and edge energy leave the GEMM epilogues
WIDE = Arch(n_species=3, lmax=2, n_layers=2, channels=64, two_body=(128, 1024), latent=(1024, 1024), edge=(128,))
# three layers (pseudo-parity features in the middle layers) and l_max 3: the generic row path
L3X3 = Arch(n_species=2, lmax=3, n_layers=3, channels=16, two_body=(32,), latent=(64,), edge=(8,))
L2X3 = Arch(n_species=3, lmax=2, n_layers=3, channels=64, two_body=(32, 64), latent=(64, 64), edge=())
L3X2 = Arch(n_species=2, lmax=3, n_layers=2, channels=32, two_body=(64,), latent=(64,), edge=(16,))
# 128 channels on the generic path: four channels per lane in its warp-per-atom kernels
L3X3C128 = Arch(n_species=2, lmax=3, n_layers=3, channels=128, two_body=(64,), latent=(64,), edge=(16,))


def _cases():
    s1, a1, w1 = make_config("c1")
    st = lattice_box(300, (300 / 0.1) ** (1 / 3), seed=2)
    st.species = st.species % 3
    s2 = lattice_box(2000, (2000 / 0.1) ** (1 / 3), seed=5)
    sl = lattice_box(700, (700 / 0.1) ** (1 / 3), seed=8)
    sl.species = sl.species % 2
    s128 = lattice_box(256, (256 / 0.1) ** (1 / 3), seed=9)
    s128.species = s128.species % 2
    sd = lattice_box(400, (400 / 0.32) ** (1 / 3), seed=10)
    sd.species = sd.species % 3
    sw = lattice_box(250, (250 / 0.1) ** (1 / 3), seed=11)
    sw.species = sw.species % 3
    s3 = lattice_box(200, (200 / 0.1) ** (1 / 3), seed=12)
    s3.species = s3.species % 2
    s3b = lattice_box(240, (240 / 0.1) ** (1 / 3), seed=13)
    s3b.species = s3b.species % 3
    s3c = lattice_box(120, (120 / 0.1) ** (1 / 3), seed=14)
    s3c.species = s3c.species % 2
    return {
        "c1": (a1, w1, s1),
        "tiny2_lmax2_C8": (TINY2, make_weights(TINY2, 3), st),
        "tiny1_lmax2_C16": (TINY1, make_weights(TINY1, 4), st),
        "lmax1_two_layers": (L1X2, make_weights(L1X2, 6), sl),
        "c2arch_2000": (ARCHS["c2"], make_weights(ARCHS["c2"], 1), s2),
        "C128_lmax2": (C128, make_weights(C128, 7), s128),
        "dense_rows_85": (DENSE, make_weights(DENSE, 8), sd),
        "wide_1024": (WIDE, make_weights(WIDE, 9), sw),
        "three_layers_lmax3": (L3X3, make_weights(L3X3, 10), s3),
        "three_layers_lmax2": (L2X3, make_weights(L2X3, 11), s3b),
        "two_layers_lmax3": (L3X2, make_weights(L3X2, 12), s3),
        "three_layers_lmax3_C128": (L3X3C128, make_weights(L3X3C128, 13), s3c),
    }


CASES = _cases()


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


_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        arch, w, s = CASES[name]
        i, j, S = neighbor_list(s.pos, s.cell, s.pbc, arch.r_c)
        _ORACLE[name] = ((i, j, S), AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S))
    return _ORACLE[name]


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_matches_oracle(name):
    arch, w, s = CASES[name]
    res, edges = _run(arch, w, s, "fp32")
    eo, (E0, Ea0, F0, W0) = _oracle(name)
    assert_same_edges(edges, eo)
    err = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)
    assert err["e_rel"] < FP32_E, err
    assert err["f_max"] < FP32_F, err
    assert err["w_rel"] < FP32_W, err
    assert abs(res["E"][0] - E0) < FP32_E * max(abs(E0), np.abs(Ea0).sum()), (res["E"][0], E0)


@pytest.mark.parametrize("name", list(CASES))
def test_bf16_matches_oracle(name):
    arch, w, s = CASES[name]
    res, _ = _run(arch, w, s, "bf16")
    _, (E0, Ea0, F0, W0) = _oracle(name)
    err = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)
    assert err["f_rms"] < BF16_F_RMS, err
    assert err["f_max"] < 10 * BF16_F_RMS, err
    assert err["e_rel"] < 1e-2, err
    assert err["w_rel"] < 5e-2, err


# TF32 path (float32 storage, tcgen05 kind::tf32 GEMMs): the tensor core reads
# each float32 operand with 10 of its 23 mantissa bits (relative error up to
# 2^-10, against bf16's 2^-9 after rounding), while activations stay float32:
# a reduced-precision GEMM path like BF16, gated like it (measured at 0.6-0.9x
# of the BF16 path's error); the ordering FP32 < TF32 < BF16 is checked below.
@pytest.mark.parametrize("name", list(CASES))
def test_tf32_matches_oracle(name):
    arch, w, s = CASES[name]
    res, edges = _run(arch, w, s, "tf32")
    eo, (E0, Ea0, F0, W0) = _oracle(name)
    assert_same_edges(edges, eo)
    err = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)
    assert err["f_rms"] < BF16_F_RMS, err
    assert err["f_max"] < 10 * BF16_F_RMS, err
    assert err["e_rel"] < 1e-2, err
    assert err["w_rel"] < 5e-2, err


def test_tf32_error_between_fp32_and_bf16():
    arch, w, s = CASES["c2arch_2000"]
    _, (E0, Ea0, F0, W0) = _oracle("c2arch_2000")
    e = {}
    for prec in ("fp32", "tf32", "bf16"):
        res, _ = _run(arch, w, s, prec)
        e[prec] = errors(res["E_atom"], res["F"], res["virial"][0], Ea0, F0, W0)["f_rms"]
    assert e["fp32"] < e["tf32"] < e["bf16"], e


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_chunked_equals_single_pass(prec):
    """Rows split over many chunks (ragged tails) give bitwise the same result."""
    arch, w, s = CASES["c2arch_2000"]
    a, _ = _run(arch, w, s, prec)
    b, _ = _run(arch, w, s, prec, chunk=6000)
    for k in ("E", "E_atom", "F", "virial"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_deterministic(prec):
    arch, w, s = CASES["tiny2_lmax2_C8"]
    a, _ = _run(arch, w, s, prec)
    b, _ = _run(arch, w, s, prec)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_degenerate_systems():
    arch, w, _ = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w))
    mu = w["mu"]
    # empty
    m.neighbors(np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 10)
    out = m.energy_forces()
    assert out["E"].item() == 0.0 and out["F"].numel() == 0
    # one atom, no neighbours: E = mu_Z, F = 0
    m.neighbors(np.array([[1.0, 2.0, 3.0]]), np.array([1], np.int32), np.eye(3) * 20)
    out = m.energy_forces()
    assert out["E"].item() == pytest.approx(mu[1], abs=1e-12)
    assert torch.all(out["F"] == 0)
    # one atom in a small cell: only its own periodic images
    pos = np.array([[0.3, 0.2, 0.1]]); cell = np.eye(3) * 3.0
    m.neighbors(pos, np.array([0], np.int32), cell)
    out = m.energy_forces()
    i, j, S = neighbor_list(pos, cell, [True] * 3, 4.0)
    E0, Ea0, F0, W0 = AllegroOracle(arch, w).energy_forces(pos, [0], cell, i, j, S)
    assert abs(out["E"].item() - E0) < 1e-5 * abs(E0)
    np.testing.assert_allclose(out["F"].cpu().numpy(), 0.0, atol=1e-6)        # symmetric images
    np.testing.assert_allclose(out["virial"].cpu().numpy()[0], W0, atol=1e-5 * np.abs(W0).max())
    # isolated atoms mixed with a bonded pair, no cell
    pos = np.array([[0.0, 0, 0], [1.5, 0, 0], [20, 0, 0], [0, 20, 0]])
    m.neighbors(pos, np.array([0, 1, 1, 0], np.int32), None)
    out = m.energy_forces()
    i, j, S = neighbor_list(pos, None, [False] * 3, 4.0)
    E0, Ea0, F0, W0 = AllegroOracle(arch, w).energy_forces(pos, [0, 1, 1, 0], None, i, j, S)
    err = errors(out["E_atom"].cpu().numpy(), out["F"].cpu().numpy(), None, Ea0, F0, W0)
    assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F, err
    m.close()


def test_bad_inputs_fail_cleanly():
    from paper_2304_10061_gb300 import AllegroError
    arch, w, s = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w))
    with pytest.raises(AllegroError):
        m.energy_forces()                                    # no neighbour list yet
    with pytest.raises(AllegroError):
        m.neighbors(s.pos, np.full(64, 7, np.int32), s.cell)  # type outside the species map
    p = s.pos.copy(); p[3, 1] = np.nan
    with pytest.raises(AllegroError):
        m.neighbors(p, s.species, s.cell)
    with pytest.raises(AllegroError):
        m.neighbors(s.pos, s.species, np.zeros((3, 3)))       # singular cell
    m.neighbors(s.pos, s.species, s.cell)                     # still usable afterwards
    assert np.isfinite(m.energy_forces()["E"].item())
    m.close()


def test_fixed_capacity_reports_need():
    from paper_2304_10061_gb300 import AllegroError
    arch, w, s = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w))
    m.reserve(64, 100, fixed=True)
    with pytest.raises(AllegroError) as ei:
        m.neighbors(s.pos, s.species, s.cell)
    assert ei.value.status == 4 and "1680" in str(ei.value)
    m.reserve(64, 2000, fixed=True)
    assert m.neighbors(s.pos, s.species, s.cell) == 1680
    m.close()


def test_species_map():
    arch, w, s = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w), species_map=[1, 0, 1])
    types = np.where(s.species == 0, 1, 0).astype(np.int32)       # type 1 -> species 0, type 0 -> 1
    m.neighbors(s.pos, types, s.cell)
    a = m.energy_forces()["E"].item()
    m2 = lib_model(weights_to_blob(arch, w))
    m2.neighbors(s.pos, s.species, s.cell)
    assert a == m2.energy_forces()["E"].item()
    m.close(); m2.close()


def test_forces_match_gpu_finite_differences():
    """The adjoint against central differences of the GPU's own float64-reduced energy."""
    arch, w, s = CASES["lmax1_two_layers"]
    m = lib_model(weights_to_blob(arch, w))
    m.neighbors(s.pos, s.species, s.cell)
    F = m.energy_forces()["F"].cpu().numpy()
    h = 2e-3
    for k, ax in ((3, 0), (100, 1), (411, 2)):
        e = []
        for sg in (1, -1):
            p = s.pos.copy(); p[k, ax] += sg * h
            m.neighbors(p, s.species, s.cell)
            e.append(m.energy_forces(forces=False, virial=False)["E"].item())
        fd = -(e[0] - e[1]) / (2 * h)
        assert abs(fd - F[k, ax]) < 2e-3 * np.sqrt((F ** 2).mean()) + 1e-3 * abs(F[k, ax]), (k, ax, fd, F[k, ax])
    m.close()


def test_autograd_function_and_host_buffers():
    from paper_2304_10061_gb300 import AllegroEnergy
    arch, w, s = CASES["c1"]
    m = lib_model(weights_to_blob(arch, w))
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    E = AllegroEnergy.apply(pos, m, torch.tensor(s.species, dtype=torch.int32, device="cuda"),
                            torch.tensor(s.cell, device="cuda"))
    E.backward()
    m.neighbors(s.pos, s.species, s.cell)            # host numpy inputs
    out = {"E": np.zeros(1), "E_atom": np.zeros(64), "F": np.zeros((64, 3)), "virial": np.zeros((1, 3, 3))}
    m.energy_forces(out=out)                          # host output buffers
    assert E.item() == out["E"][0]
    np.testing.assert_array_equal(-pos.grad.cpu().numpy(), out["F"])
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batched_molecules_per_structure(prec):
    """Many uneven gas-phase molecules in one packed list: per-molecule E, F, virial."""
    arch, w = ARCHS["c2"], make_weights(ARCHS["c2"], 1)
    mols = molecule_batch(96, seed=2)
    pos, spec, offs = pack(mols)
    m = lib_model(weights_to_blob(arch, w), precision=prec)
    m.neighbors_batched(offs, pos, spec)
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    orc = AllegroOracle(arch, w)
    for b in (0, 17, 95):
        mb = mols[b]
        i, j, S = neighbor_list(mb.pos, None, mb.pbc, 4.0)
        E0, Ea0, F0, W0 = orc.energy_forces(mb.pos, mb.species, None, i, j, S)
        sl = slice(offs[b], offs[b + 1])
        err = errors(out["E_atom"][sl], out["F"][sl], out["virial"][b], Ea0, F0, W0)
        if prec == "fp32":
            assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F and err["w_rel"] < FP32_W, (b, err)
            assert abs(out["E"][b] - E0) < FP32_E * np.abs(Ea0).sum()
        else:
            assert err["f_rms"] < BF16_F_RMS, (b, err)
    m.close()
