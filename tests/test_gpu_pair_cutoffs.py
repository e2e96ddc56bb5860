"""GPU parity of per-ordered-species-pair cutoffs (Sec. "Species-dependent cutoffs";
the production table of "Training details"): the library's neighbour lists equal
the oracle's per-pair rule exactly (periodic box and packed molecules), energies,
forces and virial match the FP64 oracle (float32 path within the float32 gates,
BF16 path within its force gate), clearing the table restores the single-cutoff
model, and invalid tables are rejected."""
from dataclasses import replace

import numpy as np
import pytest

from gpu_util import BF16_F_RMS, FP32_E, FP32_F, FP32_W, assert_same_edges, errors, lib_model
from oracle.allegro import AllegroOracle
from oracle.neighbors import neighbor_list
from synth import Arch, lattice_box, make_weights, molecule_batch, paper_pair_cutoffs, weights_to_blob

pytestmark = pytest.mark.gpu

TABLE = paper_pair_cutoffs()
ARCH = Arch(n_species=5, lmax=2, n_layers=2, channels=16, two_body=(32,), latent=(32,), edge=(),
            pair_rc=TABLE)
W = make_weights(ARCH, 21)
BLOB = weights_to_blob(ARCH, W)


def _box(n=2000, seed=12):
    return lattice_box(n, (n / 0.1) ** (1 / 3), seed=seed)


def _oracle_edges(s, pair_rc=TABLE):
    return neighbor_list(s.pos, s.cell, s.pbc, 4.0, species=s.species, pair_rc=pair_rc)


def _model(prec, table=TABLE):
    m = lib_model(BLOB, precision=prec)
    m.set_pair_cutoffs(np.asarray(table) if table is not None else None)
    return m


def test_pair_neighbor_list_is_exact():
    s = _box()
    m = _model("fp32")
    m.neighbors(s.pos, s.species, s.cell)
    got = m.get_neighbors()
    m.close()
    want = _oracle_edges(s)
    assert_same_edges(got, want)
    assert want[0].size < neighbor_list(s.pos, s.cell, s.pbc, 4.0)[0].size   # the table removes edges


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_pair_cutoffs_match_oracle(prec):
    s = _box()
    m = _model(prec)
    m.neighbors(s.pos, s.species, s.cell)
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    m.close()
    E0, Ea0, F0, W0 = AllegroOracle(ARCH, W).energy_forces(s.pos, s.species, s.cell, *_oracle_edges(s))
    err = errors(out["E_atom"], out["F"], out["virial"][0], Ea0, F0, W0)
    if prec == "fp32":
        assert err["e_rel"] < FP32_E, err
        assert err["f_max"] < FP32_F, err
        assert err["w_rel"] < FP32_W, err
    else:
        assert err["f_rms"] < BF16_F_RMS, err
        assert err["e_rel"] < 1e-2, err


def test_clearing_the_table_restores_the_single_cutoff():
    s = _box(800, seed=13)
    m = _model("fp32")
    m.set_pair_cutoffs(None)
    m.neighbors(s.pos, s.species, s.cell)
    got = m.get_neighbors()
    out = {k: v.cpu().numpy() for k, v in m.energy_forces().items()}
    m.close()
    want = neighbor_list(s.pos, s.cell, s.pbc, 4.0)
    assert_same_edges(got, want)
    E0, Ea0, F0, W0 = AllegroOracle(replace(ARCH, pair_rc=None), W).energy_forces(s.pos, s.species, s.cell, *want)
    err = errors(out["E_atom"], out["F"], out["virial"][0], Ea0, F0, W0)
    assert err["e_rel"] < FP32_E and err["f_max"] < FP32_F, err


def test_pair_cutoffs_in_packed_molecules():
    mols = molecule_batch(64, seed=14)
    offs = np.cumsum([0] + [len(x.species) for x in mols]).astype(np.int64)
    pos = np.concatenate([x.pos for x in mols])
    species = np.concatenate([x.species for x in mols]).astype(np.int32)
    m = _model("fp32")
    m.neighbors_batched(offs, pos, species)
    got = m.get_neighbors()
    m.close()
    I, J, SS = [], [], []
    for k, x in enumerate(mols):
        i, j, S = neighbor_list(x.pos, x.cell, x.pbc, 4.0, species=x.species, pair_rc=TABLE)
        I.append(i + offs[k]); J.append(j + offs[k]); SS.append(S)
    assert_same_edges(got, (np.concatenate(I), np.concatenate(J), np.concatenate(SS)))


def test_invalid_tables_are_rejected():
    from paper_2304_10061_gb300 import AllegroError
    m = lib_model(BLOB, precision="fp32")
    bad = np.asarray(TABLE).copy()
    bad[0, 1] = 4.5                        # beyond the model cutoff
    with pytest.raises(AllegroError):
        m.set_pair_cutoffs(bad)
    bad[0, 1] = 0.0
    with pytest.raises(AllegroError):
        m.set_pair_cutoffs(bad)
    with pytest.raises(AllegroError):
        m.set_pair_cutoffs(np.full((4, 4), 3.0))   # wrong species count
    m.set_pair_cutoffs(np.asarray(TABLE))  # a valid table still loads
    m.close()
