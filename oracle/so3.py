"""O(3) building blocks of the oracle: real spherical harmonics, real Wigner-3j
coupling tensors, tensor-product paths and the fused path tensor.

Conventions (the paper defers them to the Allegro paper; these are the
readings this repository fixes, and the CUDA path implements them separately):

* Real spherical harmonics, component normalised (sum_m Y_lm^2 = 2l+1 on the
  unit sphere), m = -l..l, evaluated on the unit vector (x, y, z):
      Y_lm = N_l|m| * (d^|m| P_l / dz^|m|)(z) * A_m(x, y),
      A_m = Re (x+iy)^m (m>0), 1 (m=0), Im (x+iy)^|m| (m<0),
      N_lm = sqrt((2l+1) (2 - delta_m0) (l-m)! / (l+m)!).
  This is sqrt(4 pi) times the usual real harmonics built from the
  Condon-Shortley complex ones; e.g. Y_1 = sqrt(3) (y, z, x).
* Parity of Y_l is (-1)^l ("natural parity", Eq. 1 indexes irreps by (l, p)).
* Real-basis coupling tensor C(l1,l2,l3)[m1,m2,m3]: the complex
  Clebsch-Gordan tensor (Racah's formula) taken to the real basis above, made
  real, scaled to unit Frobenius norm, and signed so that its first nonzero
  entry in row-major (m1, m2, m3) order is positive.  It is the "w3j" of
  Sec. "Optimized tensor product".
* Paths (Sec. "Optimized tensor product"): (l1,p1) x (l2,p2) -> (lo,po) with
  |l1-l2| <= lo <= l1+l2 and po = p1*p2; the env features carry natural parity
  (l2, (-1)^l2).  A layer keeps only outputs that can still reach the scalar
  0e in the remaining layers ("omitting all paths ... not allowed to
  eventually contribute to the final scalar outputs"); the last layer keeps 0e
  only.  Irreps are laid out in one strided array ordered by l, then p = +1
  before p = -1.
* Path weights (Sec. "Optimized tensor product", the learned weighted sum
  over paths sharing (lo, po)): one scalar per path and layer,
  theta = raw[lo, po, l1, p1, l2] / sqrt(n_paths(lo, po)), with parity index
  0 for p = +1 and 1 for p = -1; folded with the coupling tensors into one
  constant W[a, b, c] per layer.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache
from typing import Dict, List, Tuple

import numpy as np
import torch

Irrep = Tuple[int, int]  # (l, p) with p in {+1, -1}


# --------------------------------------------------------------------------
# Real spherical harmonics
# --------------------------------------------------------------------------

@lru_cache(maxsize=None)
def _legendre_deriv_coeffs(l: int, m: int) -> Tuple[Fraction, ...]:
    """Coefficients c_k of d^m P_l / dz^m = sum_k c_k z^k (exact rationals).

    P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k, l) z^(l-2k)  (explicit Legendre sum).
    """
    P = [Fraction(0)] * (l + 1)
    for k in range(l // 2 + 1):
        P[l - 2 * k] += Fraction((-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l), 2 ** l)
    for _ in range(m):
        P = [P[k + 1] * (k + 1) for k in range(len(P) - 1)] or [Fraction(0)]
    return tuple(P)


def sh_norm(l: int, m: int) -> float:
    am = abs(m)
    return math.sqrt((2 * l + 1) * (2 - (m == 0)) * math.factorial(l - am) / math.factorial(l + am))


def real_sh(lmax: int, rhat: torch.Tensor) -> torch.Tensor:
    """Y[..., l^2 + l + m] for l <= lmax, on unit vectors rhat[..., 3] (differentiable)."""
    x, y, z = rhat[..., 0], rhat[..., 1], rhat[..., 2]
    # (x + i y)^m as (re, im) pairs, m = 0..lmax
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, lmax + 1):
        re.append(re[-1] * x - im[-1] * y)
        im.append(re[-2] * y + im[-1] * x)
    zp = [torch.ones_like(z)]
    for k in range(1, lmax + 1):
        zp.append(zp[-1] * z)
    out = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            c = _legendre_deriv_coeffs(l, am)
            q = torch.zeros_like(z)
            for k, ck in enumerate(c):
                if ck != 0:
                    q = q + float(ck) * zp[k]
            a = re[am] if m >= 0 else im[am]
            out.append(sh_norm(l, m) * q * a)
    return torch.stack(out, dim=-1)


# --------------------------------------------------------------------------
# Clebsch-Gordan (complex, Condon-Shortley) and real coupling tensors
# --------------------------------------------------------------------------

def _fact(n: int) -> int:
    return math.factorial(n)


def cg_complex(j1: int, m1: int, j2: int, m2: int, j3: int, m3: int) -> float:
    """<j1 m1 j2 m2 | j3 m3> by Racah's formula (integer j)."""
    if m1 + m2 != m3:
        return 0.0
    if not (abs(j1 - j2) <= j3 <= j1 + j2):
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    pref = Fraction((2 * j3 + 1) * _fact(j3 + j1 - j2) * _fact(j3 - j1 + j2) * _fact(j1 + j2 - j3),
                    _fact(j1 + j2 + j3 + 1))
    pref *= Fraction(_fact(j3 + m3) * _fact(j3 - m3) * _fact(j1 - m1) * _fact(j1 + m1)
                     * _fact(j2 - m2) * _fact(j2 + m2))
    s = Fraction(0)
    for k in range(0, j1 + j2 + j3 + 1):
        a = [k, j1 + j2 - j3 - k, j1 - m1 - k, j2 + m2 - k, j3 - j2 + m1 + k, j3 - j1 - m2 + k]
        if min(a) < 0:
            continue
        den = 1
        for t in a:
            den *= _fact(t)
        s += Fraction((-1) ** k, den)
    return float(s) * math.sqrt(float(pref))


def real_from_complex(l: int) -> np.ndarray:
    """U[m, mu] with Y_real = U @ Y_complex (rows/cols indexed m + l)."""
    U = np.zeros((2 * l + 1, 2 * l + 1), dtype=np.complex128)
    s = 1.0 / math.sqrt(2.0)
    for m in range(-l, l + 1):
        if m == 0:
            U[l, l] = 1.0
        elif m > 0:
            U[m + l, m + l] = (-1) ** m * s
            U[m + l, -m + l] = s
        else:
            mu = -m
            U[m + l, -mu + l] = 1j * s
            U[m + l, mu + l] = -1j * (-1) ** mu * s
    return U


@lru_cache(maxsize=None)
def coupling_tensor(l1: int, l2: int, l3: int) -> np.ndarray:
    """Real-basis coupling tensor C[m1, m2, m3] (unit Frobenius norm, sign-fixed)."""
    Tc = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            m3 = m1 + m2
            if abs(m3) <= l3:
                Tc[m1 + l1, m2 + l2, m3 + l3] = cg_complex(l1, m1, l2, m2, l3, m3)
    U1, U2, U3 = real_from_complex(l1), real_from_complex(l2), real_from_complex(l3)
    Tr = np.einsum("ai,bj,ck,ijk->abc", U1.conj(), U2.conj(), U3, Tc)
    if np.abs(Tr.imag).max() > np.abs(Tr.real).max():
        T = Tr.imag
    else:
        T = Tr.real
    T = T / np.linalg.norm(T)
    flat = T.reshape(-1)
    nz = np.nonzero(np.abs(flat) > 1e-10)[0]
    if flat[nz[0]] < 0:
        T = -T
    T[np.abs(T) < 1e-14] = 0.0
    return T


# --------------------------------------------------------------------------
# Irreps, paths and the fused path tensor
# --------------------------------------------------------------------------

def sort_irreps(irreps) -> List[Irrep]:
    return sorted(set(irreps), key=lambda lp: (lp[0], -lp[1]))


def natural_irreps(lmax: int) -> List[Irrep]:
    return [(l, (-1) ** l) for l in range(lmax + 1)]


def irrep_dim(irreps: List[Irrep]) -> int:
    return sum(2 * l + 1 for l, _ in irreps)


def irrep_offsets(irreps: List[Irrep]) -> Dict[Irrep, int]:
    off, o = {}, 0
    for l, p in irreps:
        off[(l, p)] = o
        o += 2 * l + 1
    return off


def _tp_outputs(ir_in: List[Irrep], lmax: int) -> List[Irrep]:
    out = set()
    for l1, p1 in ir_in:
        for l2, p2 in natural_irreps(lmax):
            for lo in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                out.add((lo, p1 * p2))
    return sort_irreps(out)


def _can_reach_scalar(ir: Irrep, steps: int, lmax: int) -> bool:
    if steps == 0:
        return ir == (0, 1)
    return any(_can_reach_scalar(o, steps - 1, lmax) for o in _tp_outputs([ir], lmax))


def layer_irreps(lmax: int, n_layers: int) -> List[List[Irrep]]:
    """irreps[L] of V^L for L = 0..n_layers (V^0: natural parity l <= lmax)."""
    irs = [natural_irreps(lmax)]
    for L in range(1, n_layers + 1):
        cand = _tp_outputs(irs[-1], lmax)
        keep = [ir for ir in cand if _can_reach_scalar(ir, n_layers - L, lmax)]
        irs.append(sort_irreps(keep))
    return irs


def layer_paths(ir_in: List[Irrep], ir_out: List[Irrep], lmax: int):
    """Kept paths ((l1,p1), l2, (lo,po)) of one layer."""
    paths = []
    for lo, po in ir_out:
        for l1, p1 in ir_in:
            for l2 in range(lmax + 1):
                p2 = (-1) ** l2
                if abs(l1 - l2) <= lo <= l1 + l2 and po == p1 * p2:
                    paths.append(((l1, p1), l2, (lo, po)))
    return paths


def _pidx(p: int) -> int:
    return 0 if p == 1 else 1


def fused_path_tensor(theta_raw: np.ndarray, ir_in: List[Irrep], ir_out: List[Irrep], lmax: int) -> np.ndarray:
    """W[a, b, c] = sum_paths theta_path C(l1,l2,lo)[m1, m2, mo]  (float64)."""
    paths = layer_paths(ir_in, ir_out, lmax)
    n_into = {}
    for _, _, o in paths:
        n_into[o] = n_into.get(o, 0) + 1
    offi, offo = irrep_offsets(ir_in), irrep_offsets(ir_out)
    S = (lmax + 1) ** 2
    W = np.zeros((irrep_dim(ir_in), S, irrep_dim(ir_out)))
    for (l1, p1), l2, (lo, po) in paths:
        th = float(theta_raw[lo, _pidx(po), l1, _pidx(p1), l2]) / math.sqrt(n_into[(lo, po)])
        C = coupling_tensor(l1, l2, lo)
        a0, b0, c0 = offi[(l1, p1)], l2 * l2, offo[(lo, po)]
        W[a0:a0 + 2 * l1 + 1, b0:b0 + 2 * l2 + 1, c0:c0 + 2 * lo + 1] += th * C
    return W
