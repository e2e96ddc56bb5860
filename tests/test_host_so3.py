"""Host-side O(3) constants of the CUDA library against the oracle (no GPU).

The library builds the real-basis coupling tensors and the fused per-layer
path tensor of the tensor product (Sec. "Optimized tensor product") on the
host, in C++ (csrc/so3_host.cpp), independently of the oracle's construction
(oracle/so3.py).  This test compiles that host file alone with the system C++
compiler and compares, entry by entry:
  * complex Clebsch-Gordan coefficients (Racah's formula) for l <= 3;
  * real coupling tensors C(l1, l2, l3) (unit norm, sign convention) for l <= 3;
  * the fused tensors W[a][b][c] of a two-layer model (the middle layer and the
    scalar-only last layer) for l_max = 1 and 2 with seeded path weights.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import so3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2304_10061_gb300", "csrc", "so3_host.cpp")

_SHIM = r"""
#include <vector>
namespace alg {
double cg_racah(int j1, int m1, int j2, int m2, int j3, int m3);
void coupling_real(int l1, int l2, int l3, std::vector<double>& out);
void fused_layer_tensor(int lmax, const float* theta_raw, std::vector<double>& W, int& n_in, int& n_out, bool last);
}
namespace alg {
struct Irrep { int l, p; };
void layer_irreps(int lmax, int nl, std::vector<std::vector<Irrep>>& irs);
int irreps_dim(const std::vector<Irrep>& v);
void layer_tensor(int lmax, const std::vector<Irrep>& in, const std::vector<Irrep>& out, const float* theta_raw,
                  std::vector<double>& W);
}
extern "C" int t_irreps(int lmax, int nl, int L, int* lp, int cap) {
  std::vector<std::vector<alg::Irrep>> irs;
  alg::layer_irreps(lmax, nl, irs);
  const auto& v = irs[L];
  if ((int)v.size() * 2 > cap) return -1;
  for (size_t k = 0; k < v.size(); ++k) { lp[2 * k] = v[k].l; lp[2 * k + 1] = v[k].p; }
  return (int)v.size();
}
extern "C" int t_layer(int lmax, int nl, int L, const float* theta, double* out, int cap) {
  std::vector<std::vector<alg::Irrep>> irs;
  alg::layer_irreps(lmax, nl, irs);
  std::vector<double> W;
  alg::layer_tensor(lmax, irs[L - 1], irs[L], theta, W);
  if ((int)W.size() > cap) return -1;
  for (size_t i = 0; i < W.size(); ++i) out[i] = W[i];
  return (int)W.size();
}
extern "C" double t_cg(int j1, int m1, int j2, int m2, int j3, int m3) {
  return alg::cg_racah(j1, m1, j2, m2, j3, m3);
}
extern "C" int t_coupling(int l1, int l2, int l3, double* out, int cap) {
  std::vector<double> v;
  alg::coupling_real(l1, l2, l3, v);
  if ((int)v.size() > cap) return -1;
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
  return (int)v.size();
}
extern "C" int t_fused(int lmax, const float* theta, int last, double* out, int cap, int* n_in, int* n_out) {
  std::vector<double> W;
  int a = 0, c = 0;
  alg::fused_layer_tensor(lmax, theta, W, a, c, last != 0);
  if ((int)W.size() > cap) return -1;
  for (size_t i = 0; i < W.size(); ++i) out[i] = W[i];
  *n_in = a;
  *n_out = c;
  return (int)W.size();
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cxx is None or not os.path.isfile(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("needs a C++ compiler and the CUDA headers")
    d = tmp_path_factory.mktemp("so3host")
    shim = d / "shim.cpp"
    shim.write_text(_SHIM)
    so = d / "libso3host.so"
    subprocess.run([cxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", os.path.join(cuda, "include"),
                    SRC, str(shim), "-o", str(so)], check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    L.t_cg.restype = ctypes.c_double
    L.t_cg.argtypes = [ctypes.c_int] * 6
    L.t_coupling.restype = ctypes.c_int
    L.t_coupling.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    L.t_irreps.restype = ctypes.c_int
    L.t_irreps.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.t_layer.restype = ctypes.c_int
    L.t_layer.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double),
                                               ctypes.c_int]
    L.t_fused.restype = ctypes.c_int
    L.t_fused.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                          ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def test_clebsch_gordan_matches_oracle(lib):
    n = 0
    for j1 in range(4):
        for j2 in range(4):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for m1 in range(-j1, j1 + 1):
                    for m2 in range(-j2, j2 + 1):
                        m3 = m1 + m2
                        if abs(m3) > j3:
                            continue
                        ref = so3.cg_complex(j1, m1, j2, m2, j3, m3)
                        got = lib.t_cg(j1, m1, j2, m2, j3, m3)
                        assert abs(got - ref) < 1e-13, (j1, m1, j2, m2, j3, m3, got, ref)
                        n += 1
    assert n > 500
    # outside the selection rules the coefficient is zero
    assert lib.t_cg(1, 1, 1, 0, 1, 0) == 0.0
    assert lib.t_cg(1, 0, 1, 0, 3, 0) == 0.0


def test_real_coupling_tensors_match_oracle(lib):
    buf = np.zeros(7 * 7 * 7)
    for l1 in range(4):
        for l2 in range(4):
            for l3 in range(abs(l1 - l2), min(l1 + l2, 3) + 1):
                k = lib.t_coupling(l1, l2, l3, _dp(buf), buf.size)
                shape = (2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1)
                assert k == np.prod(shape)
                got = buf[:k].reshape(shape)
                ref = so3.coupling_tensor(l1, l2, l3)
                np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12, err_msg=str((l1, l2, l3)))


@pytest.mark.parametrize("lmax", [1, 2])
@pytest.mark.parametrize("last", [False, True])
def test_fused_layer_tensor_matches_oracle(lib, lmax, last):
    rng = np.random.default_rng(100 + 10 * lmax + int(last))
    lm = lmax + 1
    theta = rng.standard_normal((lm, 2, lm, 2, lm)).astype(np.float32)
    S = lm * lm
    buf = np.zeros(S * S * S)
    n_in, n_out = ctypes.c_int(), ctypes.c_int()
    k = lib.t_fused(lmax, theta.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(last), _dp(buf), buf.size,
                    ctypes.byref(n_in), ctypes.byref(n_out))
    irs = so3.layer_irreps(lmax, 2)
    ir_in = irs[0]
    ir_out = irs[2] if last else irs[1]
    assert (n_in.value, n_out.value) == (S, 1 if last else S)
    assert ir_out == ([(0, 1)] if last else so3.natural_irreps(lmax))
    got = buf[:k].reshape(S, S, n_out.value)
    ref = so3.fused_path_tensor(theta.astype(np.float64), ir_in, ir_out, lmax)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def _allowed(a: int, b: int, c: int) -> bool:
    """The coupling pattern the row kernels resolve at compile time: triangle rule with
    even l_a + l_b + l_c, |m_c| = |m_a| + |m_b| or ||m_a| - |m_b||, and the real
    harmonics' type rule (sine type, m < 0, iff exactly one factor is of sine type)."""
    la, lb, lc = (int(np.sqrt(x)) for x in (a, b, c))
    ma, mb, mc = a - la * la - la, b - lb * lb - lb, c - lc * lc - lc
    return (abs(la - lb) <= lc <= la + lb and (la + lb + lc) % 2 == 0
            and (abs(mc) == abs(ma) + abs(mb) or abs(mc) == abs(abs(ma) - abs(mb)))
            and ((mc < 0) == ((ma < 0) != (mb < 0))))


def test_sparsity_rule_is_the_oracle_pattern():
    # generic path weights: every entry the coupling allows is nonzero, and no other
    rng = np.random.default_rng(7)
    theta = rng.standard_normal((3, 2, 3, 2, 3))
    irs = so3.layer_irreps(2, 2)
    W = so3.fused_path_tensor(theta, irs[0], irs[1], 2)
    nz = np.abs(W) > 1e-12
    rule = np.array([[[_allowed(a, b, c) for c in range(9)] for b in range(9)] for a in range(9)])
    assert int(rule.sum()) == 83
    assert (nz == rule).all()


@pytest.mark.parametrize("lmax,nl", [(1, 3), (2, 3), (3, 3), (3, 2), (2, 2)])
def test_general_layer_irreps_and_tensors_match_oracle(lib, lmax, nl):
    """Irreps of every layer (pseudo-irreps in the middle layers of 3-layer models) and
    the fused tensors between them, as the host builds them, equal the oracle's."""
    irs = so3.layer_irreps(lmax, nl)
    buf = np.zeros(2 * 64, dtype=np.int32)
    for L in range(nl + 1):
        k = lib.t_irreps(lmax, nl, L, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), buf.size)
        got = [(int(buf[2 * q]), int(buf[2 * q + 1])) for q in range(k)]
        assert got == irs[L], (L, got, irs[L])
    lm = lmax + 1
    rng = np.random.default_rng(300 + 10 * lmax + nl)
    for L in range(1, nl + 1):
        theta = rng.standard_normal((lm, 2, lm, 2, lm)).astype(np.float32)
        ref = so3.fused_path_tensor(theta.astype(np.float64), irs[L - 1], irs[L], lmax)
        out = np.zeros(ref.size)
        k = lib.t_layer(lmax, nl, L, theta.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(out), out.size)
        assert k == ref.size
        np.testing.assert_allclose(out.reshape(ref.shape), ref, rtol=0, atol=1e-12, err_msg=str(L))
