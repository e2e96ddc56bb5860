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


# ---------------------------------------------------------------------------
# The float32 prefilter's band edge.  Candidates farther than a bound `band`
# from r_c^2 (in squared distance) are decided in float32, those inside it by
# the exact float64 rule.  These tests put pairs at the cutoff to within the
# float64 resolution, and at r^2 = r_c^2 -+ band just inside and just outside
# the band, in the 218.9 A box where float32 rounding of coordinates is
# largest, across box faces too, and compare bit-exactly with brute force.
# ---------------------------------------------------------------------------
import math
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BOX = 218.9


def _band(L, rc):
    """The library's bound for a periodic cube of side L with a stencil of one
    cell: per-component float32 error 8 ulp of the largest wrapped coordinate
    plus image offset (3 L + 3 L), squared-distance error from it, factor 4."""
    delta = 8.0 * (6.0 * L) * 2.0 ** -23
    return float(np.float32(4.0 * (2.0 * math.sqrt(3.0) * rc * delta + 3.0 * delta * delta + 1e-6 * rc * rc)))


def _planted_pairs(rcs, seed, band):
    """Pairs on a 31 A anchor grid whose separations sit at a cutoff:
    r = rc (1 + k 2^-52) near the origin (exact in float64), r = rc + m ulp(x)
    along an axis at large coordinates, r^2 = rc^2 -+ band (1 -+ 1e-2) in random
    directions, and pairs across each box face (the second atom wrapped).
    `rcs`: list of (rc, species_a, species_b); returns positions and species."""
    rng = np.random.default_rng(seed)
    sp = BOX / 7.0
    # general anchors: a 7^3 grid without its x < 31 A layer, which holds the
    # near-origin anchors (a 14 x 14 grid on the plane x = 0.5)
    sites = [(p, q, r) for p in range(1, 7) for q in range(7) for r in range(7)]
    rng.shuffle(sites)
    plane = [(q, r) for q in range(14) for r in range(14)]
    rng.shuffle(plane)
    pos, spec = [], []
    it, itp = iter(sites), iter(plane)
    used = set()

    def add(a, b, za, zb):
        pos.extend([a, b]); spec.extend([za, zb])

    for rc, za, zb in rcs:
        for k in range(-8, 9):                        # exact near the origin: a = (0.5, y, z)
            q, r = next(itp)
            a = np.array([0.5, q * sp / 2 + 0.25, r * sp / 2 + 0.25])
            d = rc * (1.0 + k * 2.0 ** -52)
            add(a, a + np.array([d, 0.0, 0.0]), za, zb)
        for m in range(-8, 9):                        # coordinate resolution far from the origin
            p, q, r = next(it)
            a = np.array([min(p * sp + 20.0, BOX - rc - 1.0), q * sp + 3.0, r * sp + 1.0])
            ulp = np.spacing(a[0] + rc)
            b = a.copy(); b[0] = (a[0] + rc) + m * ulp
            add(a, b, za, zb)
        for sgn in (-1.0, 1.0):                       # either side of the band's two edges
            for edge in (-1.0, 1.0):
                for f in (1.0 - 1e-2, 1.0 + 1e-2):
                    p, q, r = next(it)
                    a = np.array([p, q, r]) * sp + rng.uniform(5.0, 10.0, 3)
                    u = rng.normal(size=3); u /= np.linalg.norm(u)
                    r2 = rc * rc + edge * band * f if sgn > 0 else rc * rc + edge * band * f * 0.5
                    add(a, a + math.sqrt(r2) * u, za, zb)
        for ax in range(3):                           # across each face, second atom wrapped
            for k in (-2, 0, 2):
                while True:                           # a site whose other two coordinates are unused on this face
                    p, q, r = next(it)
                    key = (ax,) + tuple(x for n, x in enumerate((p, q, r)) if n != ax)
                    if key not in used:
                        used.add(key)
                        break
                a = np.array([p, q, r]) * sp + 7.0
                a[ax] = BOX - 0.5 * rc
                b = a.copy(); b[ax] = a[ax] + rc * (1.0 + k * 2.0 ** -52) - BOX
                add(a, b, za, zb)
    return np.array(pos), np.array(spec, np.int32)


def test_golden_dimer_strict_cutoff_through_the_library():
    """The hand-enumerated strict-cutoff dimer (pairs at exactly 4 A excluded at
    r_c = 4, included at r_c = 4.5), single and batched entry points."""
    from dataclasses import replace
    rows = [l.split() for l in open(os.path.join(GOLDEN, "neighbors_dimer.txt")) if l[0] in "AB"]
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    cell = np.eye(3) * 5.0
    for case, rc in (("A", 4.0), ("B", 4.5)):
        exp = np.array([[int(v) for v in r[1:]] for r in rows if r[0] == case])
        arch = replace(ARCHS["c1"], r_c=rc)
        m = lib_model(weights_to_blob(arch, make_weights(arch, 0)))
        m.neighbors(pos, np.zeros(2, np.int32), cell)
        assert_same_edges(m.get_neighbors(), (exp[:, 0], exp[:, 1], exp[:, 2:]))
        m.neighbors_batched(np.array([0, 2, 4]), np.concatenate([pos, pos]), np.zeros(4, np.int32),
                            np.stack([cell, cell]))
        i, j, S = m.get_neighbors()
        want = (np.concatenate([exp[:, 0], exp[:, 0] + 2]), np.concatenate([exp[:, 1], exp[:, 1] + 2]),
                np.concatenate([exp[:, 2:], exp[:, 2:]]))
        assert_same_edges((i, j, S), want)
        m.close()


@pytest.mark.parametrize("band", [_band(BOX, 4.0)], ids=lambda b: f"band={b:.6g}A2")
def test_band_edge_single_cutoff(model, band):
    from oracle.neighbors import brute_force
    pos, spec = _planted_pairs([(4.0, 0, 1), (4.0, 1, 1)], seed=3, band=band)
    cell = np.eye(3) * BOX
    model.neighbors(pos, spec, cell)
    assert_same_edges(model.get_neighbors(), brute_force(pos, cell, [True] * 3, 4.0))


@pytest.mark.parametrize("band", [_band(BOX, 4.0)], ids=lambda b: f"band={b:.6g}A2")
def test_band_edge_pair_cutoffs(band):
    """The same probes at each distinct entry of the paper's per-pair table."""
    from oracle.neighbors import brute_force
    from synth import paper_pair_cutoffs
    arch = ARCHS["c2"]
    table = paper_pair_cutoffs(default=arch.r_c)
    H, O, C = 0, 1, 2
    probes = [(3.0, H, H), (1.25, H, C), (1.25, H, O), (3.0, O, H), (4.0, C, H), (4.0, O, O)]
    pos, spec = _planted_pairs(probes, seed=4, band=band)
    cell = np.eye(3) * BOX
    m = lib_model(weights_to_blob(arch, make_weights(arch, 1)))
    m.set_pair_cutoffs(table)
    m.neighbors(pos, spec, cell)
    assert_same_edges(m.get_neighbors(), brute_force(pos, cell, [True] * 3, arch.r_c, species=spec,
                                                     pair_rc=table))
    m.close()
