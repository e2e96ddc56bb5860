"""Spatial decomposition of a periodic box into slabs with ghost halos (test
harness for the strict locality of Sec. "Optimized LAMMPS-Kokkos
implementation": each sub-domain evaluates its own atoms as centres, with
copies of the atoms within r_c of it as neighbour-only ghosts).

`slabs` splits the box along one cell axis into P slabs by fractional
coordinate; a slab's ghosts are the atoms (including the slab's own atoms'
periodic images) whose fractional coordinate along the axis lies within
r_c / w (w the perpendicular width of the cell along the axis) of the slab,
each carried with the integer image shift that places it next to the slab.
The decomposed axis is evaluated without periodicity (the ghosts stand in for
it), the other axes keep the cell's periodicity."""
import math

import numpy as np


def widths(cell):
    a, b, c = np.asarray(cell, dtype=np.float64)
    vol = abs(float(np.dot(a, np.cross(b, c))))
    return np.array([vol / np.linalg.norm(np.cross(b, c)), vol / np.linalg.norm(np.cross(c, a)),
                     vol / np.linalg.norm(np.cross(a, b))])


def slabs(pos, cell, P, r_c, axis=0):
    """[(local index array, ghost index array, ghost image shift array)] for P slabs."""
    cell = np.asarray(cell, dtype=np.float64)
    frac = np.asarray(pos, dtype=np.float64) @ np.linalg.inv(cell)
    f = frac[:, axis] - np.floor(frac[:, axis])          # in [0, 1)
    f = np.where(f >= 1.0, 0.0, f)
    m = r_c / widths(cell)[axis] * (1.0 + 1e-6) + 1e-9   # halo depth in fractional units
    reach = int(math.ceil(m)) + 1
    out = []
    for k in range(P):
        lo, hi = k / P, (k + 1) / P
        local = np.nonzero((f >= lo) & (f < hi))[0]
        g_idx, g_shift = [], []
        for s in range(-reach, reach + 1):
            fs = f + s                                   # fractional coordinate of the atom's image s
            near = (fs >= lo - m) & (fs < hi + m)
            if s == 0:
                near &= ~((f >= lo) & (f < hi))
            idx = np.nonzero(near)[0]
            g_idx.append(idx)
            g_shift.append(np.full(idx.size, s, dtype=np.int64))
        out.append((local, np.concatenate(g_idx), np.concatenate(g_shift)))
    return out


def subdomain_positions(pos, cell, part, axis=0):
    """Positions of one sub-domain: its local atoms (wrapped onto the slab along the axis),
    then its ghosts (wrapped, plus their image shift), and the shift applied to each local atom."""
    cell = np.asarray(cell, dtype=np.float64)
    local, ghost, gshift = part
    frac = np.asarray(pos, dtype=np.float64) @ np.linalg.inv(cell)
    wrap = np.floor(frac[:, axis])
    lp = pos[local] - wrap[local, None] * cell[axis]
    gp = pos[ghost] + (gshift - wrap[ghost])[:, None] * cell[axis]
    return np.concatenate([lp, gp]), wrap
