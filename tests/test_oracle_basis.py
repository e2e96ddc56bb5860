"""Pins of the oracle's O(3) and radial building blocks against closed forms,
library special cases and symmetry (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import so3
from oracle.allegro import bessel, envelope

RNG = np.random.default_rng(1234)


def _unit(n):
    v = RNG.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _rotation(seed, reflect=False):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return -q if reflect else q


def test_real_sh_matches_scipy_complex_harmonics():
    """Library special case: scipy's complex Y_l^m (Condon-Shortley) taken to the
    real basis and scaled by sqrt(4 pi) equals the oracle's component-normalised Y."""
    from scipy.special import sph_harm_y
    v = _unit(64)
    Y = so3.real_sh(4, torch.tensor(v)).numpy()
    th, ph = np.arccos(v[:, 2]), np.arctan2(v[:, 1], v[:, 0])
    for l in range(5):
        for m in range(-l, l + 1):
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * sph_harm_y(l, m, th, ph).real
            elif m == 0:
                ref = sph_harm_y(l, 0, th, ph).real
            else:
                ref = math.sqrt(2) * (-1) ** m * sph_harm_y(l, -m, th, ph).imag
            np.testing.assert_allclose(Y[:, l * l + l + m], math.sqrt(4 * math.pi) * ref, atol=1e-12)


def test_real_sh_closed_forms_and_normalisation():
    v = _unit(32)
    x, y, z = v.T
    Y = so3.real_sh(2, torch.tensor(v)).numpy()
    s3, s15, s5 = math.sqrt(3), math.sqrt(15), math.sqrt(5)
    ref = np.stack([np.ones_like(x), s3 * y, s3 * z, s3 * x, s15 * x * y, s15 * y * z,
                    s5 / 2 * (3 * z * z - 1), s15 * x * z, s15 / 2 * (x * x - y * y)], 1)
    np.testing.assert_allclose(Y, ref, atol=1e-13)
    Y4 = so3.real_sh(4, torch.tensor(v)).numpy()
    for l in range(5):
        np.testing.assert_allclose((Y4[:, l * l:(l + 1) ** 2] ** 2).sum(1), 2 * l + 1, atol=1e-12)


def _wigner_D(l, R):
    """Numerical Wigner-D in the oracle's real basis: Y_l(R r) = D Y_l(r)."""
    P = _unit(200)
    A = so3.real_sh(l, torch.tensor(P)).numpy()[:, l * l:(l + 1) ** 2]
    B = so3.real_sh(l, torch.tensor(P @ R.T)).numpy()[:, l * l:(l + 1) ** 2]
    X, *_ = np.linalg.lstsq(A, B, rcond=None)
    return X.T


@pytest.mark.parametrize("reflect", [False, True])
def test_sh_equivariance_and_parity(reflect):
    R = _rotation(7, reflect)
    v = _unit(16)
    for l in range(4):
        D = _wigner_D(l, _rotation(7, False))
        Y = so3.real_sh(l, torch.tensor(v)).numpy()[:, l * l:]
        YR = so3.real_sh(l, torch.tensor(v @ R.T)).numpy()[:, l * l:]
        sign = (-1) ** l if reflect else 1
        np.testing.assert_allclose(YR, sign * Y @ D.T, atol=1e-10)


def test_cg_matches_sympy():
    """Library special case: Racah formula vs sympy's Clebsch-Gordan."""
    wig = pytest.importorskip("sympy.physics.wigner")
    for (j1, j2, j3) in [(1, 1, 0), (1, 1, 1), (1, 1, 2), (2, 1, 1), (2, 2, 2), (3, 2, 1), (2, 2, 4)]:
        for m1 in range(-j1, j1 + 1):
            for m2 in range(-j2, j2 + 1):
                m3 = m1 + m2
                if abs(m3) > j3:
                    continue
                ref = float(wig.clebsch_gordan(j1, j2, j3, m1, m2, m3))
                assert abs(so3.cg_complex(j1, m1, j2, m2, j3, m3) - ref) < 1e-13


def test_coupling_closed_forms():
    """C(l,l,0) = delta/sqrt(2l+1); C(0,l,l) = delta/sqrt(2l+1); C(1,1,1) = +-eps/sqrt(6)
    in the (y, z, x) component order of Y_1."""
    for l in range(4):
        C = so3.coupling_tensor(l, l, 0)[:, :, 0]
        np.testing.assert_allclose(C, np.eye(2 * l + 1) / math.sqrt(2 * l + 1), atol=1e-14)
        C = so3.coupling_tensor(0, l, l)[0]
        np.testing.assert_allclose(C, np.eye(2 * l + 1) / math.sqrt(2 * l + 1), atol=1e-14)
    C = so3.coupling_tensor(1, 1, 1)
    eps = np.zeros((3, 3, 3))
    for a, b, c in [(0, 1, 2), (1, 2, 0), (2, 0, 1)]:
        eps[a, b, c], eps[b, a, c] = 1, -1
    # components (y, z, x): relabel eps over (x, y, z) to that order
    perm = [1, 2, 0]
    eps_yzx = eps[np.ix_(perm, perm, perm)]
    assert np.allclose(C, eps_yzx / math.sqrt(6)) or np.allclose(C, -eps_yzx / math.sqrt(6))


@pytest.mark.parametrize("reflect", [False, True])
def test_coupling_equivariance(reflect):
    R0 = _rotation(11)
    for l1 in range(4):
        for l2 in range(4):
            for l3 in range(abs(l1 - l2), min(l1 + l2, 4) + 1):
                C = so3.coupling_tensor(l1, l2, l3)
                x, y = RNG.normal(size=2 * l1 + 1), RNG.normal(size=2 * l2 + 1)
                D1, D2, D3 = (_wigner_D(l, R0) for l in (l1, l2, l3))
                z = np.einsum("abc,a,b->c", C, x, y)
                p1, p2 = ((-1) ** l1, (-1) ** l2) if reflect else (1, 1)
                zr = np.einsum("abc,a,b->c", C, p1 * D1 @ x, p2 * D2 @ y)
                np.testing.assert_allclose(zr, p1 * p2 * (D3 @ z), atol=1e-10)


def test_layer_irreps_and_paths():
    irs = so3.layer_irreps(2, 2)
    assert irs == [[(0, 1), (1, -1), (2, 1)]] * 2 + [[(0, 1)]]
    assert len(so3.layer_paths(irs[0], irs[1], 2)) == 11
    assert len(so3.layer_paths(irs[1], irs[2], 2)) == 3
    irs1 = so3.layer_irreps(1, 1)
    assert irs1 == [[(0, 1), (1, -1)], [(0, 1)]]
    assert len(so3.layer_paths(irs1[0], irs1[1], 1)) == 2
    # three layers: pseudo-irreps appear in the middle (e.g. 1 x 1 -> 1e), 0o never does
    irs3 = so3.layer_irreps(3, 3)
    assert (1, 1) in irs3[1] and (0, -1) not in irs3[1]
    assert irs3[2] == so3.natural_irreps(3)


def test_fused_tensor_equals_sum_of_paths():
    """Sec. 'Optimized tensor product': the fused tensor applied once equals the sum
    over paths of theta * (per-path coupling) -- computed here path by path."""
    lmax = 2
    irs = so3.layer_irreps(lmax, 2)
    theta = RNG.normal(size=(3, 2, 3, 2, 3))
    W = so3.fused_path_tensor(theta, irs[0], irs[1], lmax)
    x, g = RNG.normal(size=9), RNG.normal(size=9)
    got = np.einsum("abc,a,b->c", W, x, g)
    ref = np.zeros(9)
    counts = {}
    for (l1, p1), l2, (lo, po) in so3.layer_paths(irs[0], irs[1], lmax):
        counts[(lo, po)] = counts.get((lo, po), 0) + 1
    for (l1, p1), l2, (lo, po) in so3.layer_paths(irs[0], irs[1], lmax):
        th = theta[lo, 0 if po == 1 else 1, l1, 0 if p1 == 1 else 1, l2] / math.sqrt(counts[(lo, po)])
        ref[lo * lo:(lo + 1) ** 2] += th * np.einsum(
            "abc,a,b->c", so3.coupling_tensor(l1, l2, lo), x[l1 * l1:(l1 + 1) ** 2], g[l2 * l2:(l2 + 1) ** 2])
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_bessel_closed_forms():
    rc = 4.0
    r = torch.tensor([rc / 2, rc / 4], dtype=torch.float64)
    B = bessel(r, rc, 8).numpy()
    for n in range(1, 9):
        assert abs(B[0, n - 1] - math.sqrt(2 / rc) * math.sin(n * math.pi / 2) / (rc / 2)) < 1e-14
        assert abs(B[1, n - 1] - math.sqrt(2 / rc) * math.sin(n * math.pi / 4) / (rc / 4)) < 1e-14
    # orthonormality of r*B_n on [0, r_c] (the radial Bessel basis)
    rr = np.linspace(1e-9, rc, 200001)
    Bn = bessel(torch.tensor(rr), rc, 4).numpy() * rr[:, None]
    G = (Bn[:, :, None] * Bn[:, None, :]).sum(0) * (rr[1] - rr[0])
    np.testing.assert_allclose(G, np.eye(4), atol=1e-4)


def test_envelope_closed_form_and_smoothness():
    x = torch.tensor([0.0, 0.5, 1.0, 1.2], dtype=torch.float64, requires_grad=True)
    u = envelope(x, 6)
    xv = x.detach().numpy()
    ref = 1 - 28 * xv ** 6 + 48 * xv ** 7 - 21 * xv ** 8
    ref[3] = 0.0
    np.testing.assert_allclose(u.detach().numpy(), ref, atol=1e-14)
    assert u[0].item() == 1.0 and abs(u[2].item()) < 1e-14
    g, = torch.autograd.grad(u.sum(), x, create_graph=True)
    gg, = torch.autograd.grad(g.sum(), x)
    assert abs(g[2].item()) < 1e-12 and abs(gg[2].item()) < 1e-10
