"""GPU neighbour lists vs the oracle's rule: bit-exact (i, j, S) sets."""
import numpy as np
import pytest

from gpu_util import assert_same_edges, lib_model
from oracle.neighbors import neighbor_list, neighbor_list_batched
from synth import ARCHS, make_weights, weights_to_blob, lattice_box, random_box, molecule_batch, make_config
from synth.structures import pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    arch = ARCHS["c1"]
    m = lib_model(weights_to_blob(arch, make_weights(arch, 0)))
    yield m
    m.close()


def _check(m, pos, types, cell, pbc):
    m.neighbors(pos, types, cell, None if pbc is None else np.asarray(pbc, np.uint8))
    want = neighbor_list(pos, cell, [True] * 3 if pbc is None and cell is not None else
                         (pbc if pbc is not None else [False] * 3), 4.0)
    assert_same_edges(m.get_neighbors(), want)
    return len(want[0])


def test_c1_box(model):
    s = random_box(64, 8.62, seed=0)
    assert _check(model, s.pos, s.species, s.cell, None) > 0


@pytest.mark.parametrize("n", [500, 2000, 23552])
def test_lattice_boxes(model, n):
    s = lattice_box(n, (n / 0.1) ** (1 / 3), seed=n)
    _check(model, s.pos, s.species % 2, s.cell, None)


@pytest.mark.parametrize("pbc", [[1, 1, 1], [1, 0, 1], [0, 1, 0], [0, 0, 0]])
def test_triclinic_unwrapped(model, pbc):
    rng = np.random.default_rng(5)
    cell = np.array([[6.0, 0.0, 0.0], [2.1, 5.5, 0.0], [-1.3, 1.7, 7.2]])
    pos = rng.uniform(-0.2, 1.2, (40, 3)) @ cell
    _check(model, pos, np.zeros(40, np.int32), cell, pbc)


def test_thin_cell_self_images(model):
    rng = np.random.default_rng(1)
    cell = np.diag([2.5, 3.0, 9.0])
    pos = rng.uniform(0, 1, (5, 3)) @ cell
    n = _check(model, pos, np.zeros(5, np.int32), cell, [1, 1, 1])
    i, j, S = model.get_neighbors()
    assert n > 0 and np.any((i == j) & np.any(S != 0, axis=1))


def test_single_atom_and_empty(model):
    cell = np.eye(3) * 3.0
    assert _check(model, np.array([[0.5, 0.5, 0.5]]), np.zeros(1, np.int32), cell, [1, 1, 1]) == 6
    assert _check(model, np.array([[0.5, 0.5, 0.5]]), np.zeros(1, np.int32), np.eye(3) * 20, [1, 1, 1]) == 0
    assert model.neighbors(np.zeros((0, 3)), np.zeros(0, np.int32), np.eye(3) * 10) == 0


def test_isolated_atoms_nonperiodic(model):
    pos = np.array([[0.0, 0, 0], [10.0, 0, 0], [0, 10.0, 0], [0, 0, 3.9], [30, 30, 30]])
    _check(model, pos, np.zeros(5, np.int32), None, [0, 0, 0])


def test_gpu_inputs_on_device(model):
    import torch
    s = lattice_box(1000, (1000 / 0.1) ** (1 / 3), seed=4)
    model.neighbors(torch.tensor(s.pos, device="cuda"), torch.tensor(s.species % 2, dtype=torch.int32,
                                                                     device="cuda"),
                    torch.tensor(s.cell, device="cuda"))
    assert_same_edges(model.get_neighbors(), neighbor_list(s.pos, s.cell, s.pbc, 4.0))


def test_batched_molecules(model):
    mols = molecule_batch(200, seed=2)
    pos, spec, offs = pack(mols)
    model.neighbors_batched(offs, pos, spec % 2)
    assert_same_edges(model.get_neighbors(), neighbor_list_batched(mols, 4.0))


def test_batched_periodic_boxes(model):
    boxes = [lattice_box(n, (n / 0.1) ** (1 / 3), seed=n) for n in (30, 64, 100)]
    pos, spec, offs = pack(boxes)
    cells = np.stack([b.cell for b in boxes])
    model.neighbors_batched(offs, pos, spec % 2, cells)
    assert_same_edges(model.get_neighbors(), neighbor_list_batched(boxes, 4.0))


def test_rows_sorted_and_deterministic(model):
    s = lattice_box(3000, (3000 / 0.1) ** (1 / 3), seed=7)
    model.neighbors(s.pos, s.species % 2, s.cell)
    a = model.get_neighbors()
    model.neighbors(s.pos, s.species % 2, s.cell)
    b = model.get_neighbors()
    assert np.all(np.diff(a[0]) >= 0)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_c4_sampled_rows(model):
    """Full 1,048,576-atom box: sampled centre rows equal the oracle's rows."""
    s, _, _ = make_config("c4")
    model.neighbors(s.pos, s.species % 2, s.cell)
    i, j, S = model.get_neighbors()
    assert model.n_edges > 24 * s.n_atoms
    cs = np.random.default_rng(0).choice(s.n_atoms, 48, replace=False)
    want = neighbor_list(s.pos, s.cell, s.pbc, 4.0, centers=np.sort(cs))
    m = np.isin(i, cs)
    assert_same_edges((i[m], j[m], S[m]), want)
