"""Ordered neighbour pairs within the cutoff (FP64, numpy).

Definition (Sec. "Allegro": E_i = sum over j in N(i) of ordered-pair
energies; Sec. "Species-dependent cutoffs": pairs are ordered).  An edge is a
triple (i, j, S) with S in Z^3 an image shift (S_k = 0 on non-periodic axes)
and displacement evaluated componentwise, in exactly this order and with no
fused multiply-add:
    off[x] = (S0*a[x] + S1*b[x]) + S2*c[x]
    d[x]   = (pos_j[x] + off[x]) - pos_i[x]
    r2     = (d[0]*d[0] + d[1]*d[1]) + d[2]*d[2]
and the edge exists iff r2 < r_c*r_c (strict) and not (i == j and S == 0).
Periodic self-images (i == j, S != 0) are edges when within the cutoff.
S ranges over |S_k| <= ceil(r_c / w_k + span_k), w_k the perpendicular width
of the cell along axis k and span_k the spread of the atoms' fractional
coordinates along k (positions need not be wrapped into the cell; for wrapped
positions this is the usual ceil(r_c / w_k) plus one layer, which adds
candidates, never edges).  numpy evaluates elementwise float64 operations without
contraction, so the arithmetic above is what runs.

Per-ordered-species-pair cutoffs (Sec. "Species-dependent cutoffs"): with a
table pair_rc[Z_i][Z_j] (row = centre species) the test is r2 < rc*rc with
rc = pair_rc[Z_i][Z_j] for the candidate's ordered pair, every other part of
the rule unchanged; the image range uses the largest entry.

`brute_force` is the definition, applied to every candidate.
`neighbor_list` applies the same test to a superset of candidates found with
a k-d tree at radius r_c (1 + 1e-6) + 1e-9; it is checked against
`brute_force` in the tests and used for inputs too large for brute force.
Output: int64 arrays i, j and int64 S[E, 3], sorted by (i, j, S0, S1, S2).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def _widths(cell: np.ndarray) -> np.ndarray:
    a, b, c = cell
    vol = abs(float(np.dot(a, np.cross(b, c))))
    return np.array([vol / np.linalg.norm(np.cross(b, c)),
                     vol / np.linalg.norm(np.cross(c, a)),
                     vol / np.linalg.norm(np.cross(a, b))])


def image_range(cell, pbc, r_c, pos=None):
    if cell is None:
        return [0, 0, 0]
    cell = np.asarray(cell, dtype=np.float64)
    w = _widths(cell)
    span = np.zeros(3)
    if pos is not None and len(pos) > 1:
        frac = np.asarray(pos, dtype=np.float64) @ np.linalg.inv(cell)
        span = frac.max(0) - frac.min(0)
    return [int(math.ceil(r_c / w[k] + span[k])) if pbc[k] else 0 for k in range(3)]


def _images(cell, pbc, r_c, pos=None):
    n = image_range(cell, pbc, r_c, pos)
    return [S for S in itertools.product(*[range(-n[k], n[k] + 1) for k in range(3)])]


def _offset(cell, S):
    if cell is None:
        return np.zeros(3)
    cell = np.asarray(cell, dtype=np.float64)
    return (float(S[0]) * cell[0] + float(S[1]) * cell[1]) + float(S[2]) * cell[2]


def _exact_test(pos, i, j, S, off, rc2):
    d = (pos[j] + off) - pos[i]
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    self_pair = (i == j) & np.all(S == 0, axis=1)
    return (r2 < rc2) & ~self_pair


def _sort(i, j, S):
    order = np.lexsort((S[:, 2], S[:, 1], S[:, 0], j, i))
    return i[order], j[order], S[order]


def _pair_rc2(species, pair_rc, ii, jj):
    """Squared cutoff of each candidate's ordered (centre, neighbour) species pair."""
    t = np.asarray(pair_rc, dtype=np.float64)
    z = np.asarray(species, dtype=np.int64)
    rc = t[z[ii], z[jj]]
    return rc * rc


def brute_force(pos, cell, pbc, r_c, centers=None, species=None, pair_rc=None):
    """Every (i, j, S) candidate tested with the exact FP64 rule (per ordered
    species pair when `pair_rc` is given; `r_c` is then its largest entry)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    centers = np.arange(n) if centers is None else np.asarray(centers, dtype=np.int64)
    if pair_rc is not None:
        r_c = float(np.max(np.asarray(pair_rc, dtype=np.float64)))
    rc2 = float(r_c) * float(r_c)
    I, J, SS = [], [], []
    for S in _images(cell, pbc, r_c, pos):
        off = _offset(cell, S)
        ii = np.repeat(centers, n)
        jj = np.tile(np.arange(n), len(centers))
        Sa = np.tile(np.array(S, dtype=np.int64), (ii.size, 1))
        keep = _exact_test(pos, ii, jj, Sa, off, rc2 if pair_rc is None else _pair_rc2(species, pair_rc, ii, jj))
        I.append(ii[keep]); J.append(jj[keep]); SS.append(Sa[keep])
    i = np.concatenate(I).astype(np.int64)
    j = np.concatenate(J).astype(np.int64)
    S = np.concatenate(SS).astype(np.int64).reshape(-1, 3)
    return _sort(i, j, S)


def neighbor_list(pos, cell, pbc, r_c, centers=None, species=None, pair_rc=None):
    """Same result as `brute_force`, with k-d tree candidate pruning."""
    from scipy.spatial import cKDTree

    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    centers = np.arange(n) if centers is None else np.asarray(centers, dtype=np.int64)
    if n == 0 or centers.size == 0:
        return (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3), np.int64))
    if pair_rc is not None:
        r_c = float(np.max(np.asarray(pair_rc, dtype=np.float64)))
    rc2 = float(r_c) * float(r_c)
    rad = float(r_c) * (1.0 + 1e-6) + 1e-9
    lo = pos[centers].min(0) - rad
    hi = pos[centers].max(0) + rad
    pts, src, shf = [], [], []
    for S in _images(cell, pbc, r_c, pos):
        off = _offset(cell, S)
        q = pos + off
        m = np.all((q >= lo) & (q <= hi), axis=1)
        idx = np.nonzero(m)[0]
        pts.append(q[idx]); src.append(idx)
        shf.append(np.tile(np.array(S, dtype=np.int64), (idx.size, 1)))
    pts = np.concatenate(pts); src = np.concatenate(src); shf = np.concatenate(shf).reshape(-1, 3)
    tree = cKDTree(pts)
    lists = tree.query_ball_point(pos[centers], rad)
    cnt = np.array([len(l) for l in lists], dtype=np.int64)
    ii = np.repeat(centers, cnt)
    cand = np.concatenate([np.asarray(l, dtype=np.int64) for l in lists]) if cnt.sum() else np.zeros(0, np.int64)
    jj = src[cand]
    Sa = shf[cand]
    cell_arr = np.zeros((3, 3)) if cell is None else np.asarray(cell, dtype=np.float64)
    off = (Sa[:, 0:1].astype(np.float64) * cell_arr[0] + Sa[:, 1:2].astype(np.float64) * cell_arr[1]) \
        + Sa[:, 2:3].astype(np.float64) * cell_arr[2]
    keep = _exact_test(pos, ii, jj, Sa, off, rc2 if pair_rc is None else _pair_rc2(species, pair_rc, ii, jj))
    return _sort(ii[keep], jj[keep], Sa[keep])


def neighbor_list_batched(structs, r_c):
    """Packed edges over independent structures: global atom indices, S per edge."""
    I, J, SS = [], [], []
    base = 0
    for s in structs:
        i, j, S = neighbor_list(s.pos, s.cell, s.pbc, r_c)
        I.append(i + base); J.append(j + base); SS.append(S)
        base += s.n_atoms
    return np.concatenate(I), np.concatenate(J), np.concatenate(SS).reshape(-1, 3)
