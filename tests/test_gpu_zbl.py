"""GPU parity of the ZBL repulsion (Sec. "Training details": the production
potential carries a ZBL term; the readings are those of the oracle's
`oracle/zbl.py`): energies, per-atom energies, forces and virial with the term
on match the FP64 oracle (float32 path within the float32 gates, BF16 path
within its force gate), single cutoff and the per-pair cutoff table, a
batched set of molecules, close contacts where the term dominates, removing
the term restores the plain model, and bad tables are rejected."""
from dataclasses import replace

import numpy as np
import pytest

from gpu_util import BF16_F_RMS, FP32_E, FP32_F, FP32_W, errors, lib_model
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from synth import (Arch, SPECIES_Z, lattice_box, make_weights, molecule_batch, paper_pair_cutoffs,
                   weights_to_blob)

pytestmark = pytest.mark.gpu

ARCH = Arch(n_species=5, lmax=2, n_layers=2, channels=16, two_body=(32,), latent=(32,), edge=(8,),
            zbl_z=SPECIES_Z)
W = make_weights(ARCH, 23)
BLOB = weights_to_blob(ARCH, W)


def _box(n=1500, seed=41, squeeze=True):
    s = lattice_box(n, (n / 0.1) ** (1 / 3), seed=seed)
    if squeeze:   # pull a few atoms close to a neighbour (0.5-0.9 A), where the repulsion dominates
        rng = np.random.default_rng(seed)
        i, j, S = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
        for e in rng.choice(len(i), 20, replace=False):
            a, b = i[e], j[e]
            d = (s.pos[b] + S[e] @ s.cell) - s.pos[a]
            s.pos[b] = s.pos[a] + d / np.linalg.norm(d) * rng.uniform(0.5, 0.9) - S[e] @ s.cell
    return s


def _check(prec, arch, s, m):
    m.neighbors(s.pos, s.species, s.cell)
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    kw = {} if arch.pair_rc is None else dict(species=s.species, pair_rc=arch.pair_rc)
    ed = neighbor_list(s.pos, s.cell, s.pbc, 4.0, **kw)
    E0, Ea0, F0, W0 = AllegroOracle(arch, W).energy_forces(s.pos, s.species, s.cell, *ed)
    err = errors(out["E_atom"], out["F"], out["virial"][0], Ea0, F0, W0)
    if prec == "fp32":
        assert err["e_rel"] < FP32_E, err
        assert err["f_max"] < FP32_F, err
        assert err["w_rel"] < FP32_W, err
        assert abs(out["E"][0] - E0) < FP32_E * max(abs(E0), 1.0)
    else:
        assert err["f_rms"] < BF16_F_RMS, err
    return out, Ea0


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_zbl_matches_oracle(prec):
    s = _box()
    m = lib_model(BLOB, precision=prec)
    m.set_zbl(SPECIES_Z)
    out, Ea0 = _check(prec, ARCH, s, m)
    m.close()
    # the term matters here: the plain model differs by far more than the tolerance
    plain = AllegroOracle(replace(ARCH, zbl_z=None), W).energy_forces(
        s.pos, s.species, s.cell, *neighbor_list(s.pos, s.cell, s.pbc, 4.0))[1]
    assert np.abs(plain - Ea0).max() > 1.0


def test_zbl_with_pair_cutoffs():
    arch = replace(ARCH, pair_rc=paper_pair_cutoffs())
    s = _box(1200, seed=42)
    m = lib_model(BLOB, precision="fp32")
    m.set_pair_cutoffs(np.asarray(arch.pair_rc))
    m.set_zbl(SPECIES_Z)
    _check("fp32", arch, s, m)
    m.close()


def test_zbl_in_packed_molecules():
    mols = molecule_batch(48, seed=43)
    offs = np.cumsum([0] + [len(x.species) for x in mols]).astype(np.int64)
    pos = np.concatenate([x.pos for x in mols])
    species = np.concatenate([x.species for x in mols]).astype(np.int32)
    m = lib_model(BLOB, precision="fp32")
    m.set_zbl(SPECIES_Z)
    m.neighbors_batched(offs, pos, species)
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    m.close()
    orc = AllegroOracle(ARCH, W)
    for k, x in enumerate(mols[:12]):
        E0, Ea0, F0, W0 = orc.energy_forces(x.pos, x.species, None, *neighbor_list(x.pos, None, x.pbc, 4.0))
        sl = slice(offs[k], offs[k + 1])
        err = errors(out["E_atom"][sl], out["F"][sl], out["virial"][k], Ea0, F0, W0)
        assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F, (k, err)


def test_removing_zbl_restores_the_plain_model():
    s = _box(600, seed=44, squeeze=False)
    m = lib_model(BLOB, precision="fp32")
    m.set_zbl(SPECIES_Z)
    m.set_zbl(None)
    _check("fp32", replace(ARCH, zbl_z=None), s, m)
    m.close()


def test_bad_atomic_numbers_are_rejected():
    from paper_2304_10061_gb300 import AllegroError
    m = lib_model(BLOB, precision="fp32")
    with pytest.raises(AllegroError):
        m.set_zbl([1, 8, 6, 7])                 # wrong species count
    with pytest.raises(AllegroError):
        m.set_zbl([1, 8, 0, 7, 16])             # Z outside 1..118
    m.set_zbl(SPECIES_Z)
    m.close()
