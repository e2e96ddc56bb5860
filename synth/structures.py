"""Seeded synthetic atomic structures at liquid-water number density.

The paper measures on solvated biomolecules and water boxes (Sec. "Scientific
applications used to measure performance").  Those structures are not
available here, so these generators produce boxes with the same number density
(0.1 atoms per cubic Angstrom) and a water/protein-like species mix.  They
reproduce density and composition, not any item of those data sets.

All generators are deterministic functions of their seed (numpy PCG64).
Units: Angstrom.  Cells are row-major 3x3 arrays whose rows are the lattice
vectors a, b, c.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Species order used by every model here: model species index -> element.
SPECIES_NAMES = ("H", "O", "C", "N", "S")
# Atomic masses in amu, same order.
SPECIES_MASSES = (1.008, 15.999, 12.011, 14.007, 32.06)
SPECIES_Z = (1, 8, 6, 7, 16)   # atomic numbers of SPECIES_NAMES
def paper_pair_cutoffs(names=None, default: float = 4.0):
    """Per-ordered-species-pair cutoffs of the paper's production model (Sec. "Training
    details"): H-H 3.0, H-C 1.25, H-O 1.25, O-H 3.0 Angstrom, every other ordered pair
    `default`.  Row = centre species, column = neighbour species, so H-C (an H centre
    with a C neighbour) is 1.25 while C-H keeps the default."""
    names = SPECIES_NAMES if names is None else tuple(names)
    special = {("H", "H"): 3.0, ("H", "C"): 1.25, ("H", "O"): 1.25, ("O", "H"): 3.0}
    return tuple(tuple(float(special.get((a, b), default)) for b in names) for a in names)


# Water / solvated-protein-like composition: H 63 %, O 30 %, C 5 %, N 1.5 %, S 0.5 %.
WATER_MIX = (0.63, 0.30, 0.05, 0.015, 0.005)


@dataclass
class Structure:
    """One structure: positions [N,3] f64, species [N] int32, cell [3,3] or None, pbc [3]."""

    pos: np.ndarray
    species: np.ndarray
    cell: Optional[np.ndarray]
    pbc: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])


def _min_image_dist2(d: np.ndarray, L: float) -> np.ndarray:
    d = d - L * np.round(d / L)
    return (d * d).sum(-1)


def random_box(n: int, L: float, seed: int, min_sep: float = 0.9,
               species_counts=(43, 21), max_tries: int = 1_000_000) -> Structure:
    """Atoms placed uniformly at random in a periodic cube, rejecting any
    candidate closer than `min_sep` (minimum image) to an accepted atom.

    Species: `species_counts[k]` atoms of species k, assigned to atom slots
    by a seeded permutation.  Draw order: all positions first, then the
    permutation.
    """
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_box: could not place atoms")
        c = rng.uniform(0.0, L, size=3)
        if k == 0 or _min_image_dist2(pos[:k] - c, L).min() >= min_sep * min_sep:
            pos[k] = c
            k += 1
    assert sum(species_counts) == n
    base = np.concatenate([np.full(c, s, dtype=np.int32) for s, c in enumerate(species_counts)])
    species = base[rng.permutation(n)].astype(np.int32)
    cell = np.diag([L, L, L]).astype(np.float64)
    return Structure(pos, species, cell, np.array([True, True, True]), name=f"random{n}",
                     meta=dict(seed=seed, L=L, min_sep=min_sep))


def _cube_root_ceil(n: int) -> int:
    m = int(round(n ** (1.0 / 3.0)))
    while m ** 3 < n:
        m += 1
    while m > 1 and (m - 1) ** 3 >= n:
        m -= 1
    return m


def lattice_box(n: int, L: float, seed: int, mix=WATER_MIX, jitter: float = 0.25) -> Structure:
    """Jittered simple-cubic lattice in a periodic cube.

    m = smallest integer with m^3 >= n sites per axis, spacing a = L/m.  n of
    the m^3 sites are chosen without replacement (kept in site order, so atom
    index order is spatially coherent), each displaced by U(-jitter*a,
    +jitter*a) per axis from the site centre; with jitter = 0.25 any two atoms
    are at least 0.5*a apart.  Species are drawn i.i.d. from `mix`.
    Draw order: site choice, jitter, species.
    """
    rng = np.random.default_rng(seed)
    m = _cube_root_ceil(n)
    a = L / m
    sites = np.sort(rng.choice(m ** 3, size=n, replace=False))
    ix, iy, iz = np.unravel_index(sites, (m, m, m))
    grid = np.stack([ix, iy, iz], axis=1).astype(np.float64)
    jit = rng.uniform(-jitter, jitter, size=(n, 3))
    pos = (grid + 0.5 + jit) * a
    p = np.asarray(mix, dtype=np.float64)
    p = p / p.sum()
    species = rng.choice(len(p), size=n, p=p).astype(np.int32)
    cell = np.diag([L, L, L]).astype(np.float64)
    return Structure(pos, species, cell, np.array([True, True, True]), name=f"lattice{n}",
                     meta=dict(seed=seed, L=L, m=m, a=a))


def molecule_batch(n_mol: int, seed: int, n_min: int = 8, n_max: int = 64,
                   bond=(1.0, 1.5), min_sep: float = 0.9, mix=WATER_MIX,
                   max_tries: int = 200) -> List[Structure]:
    """Gas-phase molecules built by a random walk.

    Each molecule has U{n_min..n_max} atoms.  Atom k+1 sits at atom k plus a
    bond of length U(bond) along a uniformly random direction; a step that
    lands closer than `min_sep` to any earlier atom of the molecule is redrawn
    (and, after `max_tries` failures, the walk restarts from a random earlier
    atom).  Species i.i.d. from `mix`.  Non-periodic: cell None, pbc all False.
    """
    rng = np.random.default_rng(seed)
    p = np.asarray(mix, dtype=np.float64)
    p = p / p.sum()
    out = []
    for mol in range(n_mol):
        n = int(rng.integers(n_min, n_max + 1))
        pos = np.zeros((n, 3))
        k = 1
        anchor = 0
        fails = 0
        while k < n:
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            c = pos[anchor] + rng.uniform(bond[0], bond[1]) * v
            d2 = ((pos[:k] - c) ** 2).sum(-1)
            if d2.min() >= min_sep * min_sep:
                pos[k] = c
                anchor = k
                k += 1
                fails = 0
            else:
                fails += 1
                if fails > max_tries:
                    anchor = int(rng.integers(0, k))
                    fails = 0
        species = rng.choice(len(p), size=n, p=p).astype(np.int32)
        out.append(Structure(pos, species, None, np.array([False, False, False]),
                             name=f"mol{mol}", meta=dict(seed=seed)))
    return out


def pack(structs: List[Structure]):
    """Concatenate structures: returns (pos [N,3], species [N], offsets [B+1] int64)."""
    offs = np.zeros(len(structs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([s.n_atoms for s in structs])
    pos = np.concatenate([s.pos for s in structs], axis=0)
    spec = np.concatenate([s.species for s in structs], axis=0).astype(np.int32)
    return pos, spec, offs
