// Host-side O(3) constants of the tensor product (Sec. "Optimized tensor product").
//
// Real-basis coupling tensors C(l1,l2,l3)[m1,m2,m3] for the real spherical
// harmonics used by the kernels (component-normalised, Y_1 ~ (y, z, x)):
// complex Clebsch-Gordan coefficients by Racah's closed formula, taken to the
// real basis, made real, scaled to unit Frobenius norm and signed so that the
// first nonzero entry in (m1, m2, m3) row-major order is positive.  The fused
// per-layer tensor is W[a][b][c] = sum over kept paths of theta_path * C,
// theta_path = raw[lo][po][l1][p1][l2] / sqrt(number of paths into (lo, po)),
// where a path is (l1, p1) x (l2, (-1)^l2) -> (lo, po = p1 (-1)^l2) with
// |l1 - l2| <= lo <= l1 + l2 (the selection rule of the paper).  For models
// with at most two layers every feature carries natural parity p = (-1)^l,
// so the strided layout index of (l, m) is l*l + l + m.
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace alg {

static double fact(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= k;
  return r;
}

double cg_racah(int j1, int m1, int j2, int m2, int j3, int m3) {
  if (m1 + m2 != m3) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  double pref = (2 * j3 + 1) * fact(j3 + j1 - j2) * fact(j3 - j1 + j2) * fact(j1 + j2 - j3) /
                fact(j1 + j2 + j3 + 1);
  pref *= fact(j3 + m3) * fact(j3 - m3) * fact(j1 - m1) * fact(j1 + m1) * fact(j2 - m2) * fact(j2 + m2);
  double s = 0.0;
  for (int k = 0; k <= j1 + j2 + j3; ++k) {
    int t[6] = {k, j1 + j2 - j3 - k, j1 - m1 - k, j2 + m2 - k, j3 - j2 + m1 + k, j3 - j1 - m2 + k};
    bool ok = true;
    double den = 1.0;
    for (int q = 0; q < 6; ++q) {
      if (t[q] < 0) { ok = false; break; }
      den *= fact(t[q]);
    }
    if (!ok) continue;
    s += ((k & 1) ? -1.0 : 1.0) / den;
  }
  return s * std::sqrt(pref);
}

// U[m][mu]: real harmonic m as a combination of complex harmonics mu.
static void real_unitary(int l, std::vector<std::complex<double>>& U) {
  const int d = 2 * l + 1;
  U.assign(d * d, 0.0);
  const double s = 1.0 / std::sqrt(2.0);
  for (int m = -l; m <= l; ++m) {
    if (m == 0) {
      U[l * d + l] = 1.0;
    } else if (m > 0) {
      U[(m + l) * d + (m + l)] = ((m & 1) ? -s : s);
      U[(m + l) * d + (-m + l)] = s;
    } else {
      int mu = -m;
      U[(m + l) * d + (-mu + l)] = std::complex<double>(0.0, s);
      U[(m + l) * d + (mu + l)] = std::complex<double>(0.0, (mu & 1) ? s : -s);
    }
  }
}

void coupling_real(int l1, int l2, int l3, std::vector<double>& out) {
  const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * l3 + 1;
  std::vector<std::complex<double>> U1, U2, U3;
  real_unitary(l1, U1);
  real_unitary(l2, U2);
  real_unitary(l3, U3);
  std::vector<std::complex<double>> T(d1 * d2 * d3, 0.0);
  for (int a = 0; a < d1; ++a)
    for (int b = 0; b < d2; ++b)
      for (int c = 0; c < d3; ++c) {
        std::complex<double> acc = 0.0;
        for (int i = 0; i < d1; ++i) {
          if (U1[a * d1 + i] == 0.0) continue;
          for (int j = 0; j < d2; ++j) {
            if (U2[b * d2 + j] == 0.0) continue;
            int k = (i - l1) + (j - l2) + l3;
            if (k < 0 || k >= d3 || U3[c * d3 + k] == 0.0) continue;
            acc += std::conj(U1[a * d1 + i]) * std::conj(U2[b * d2 + j]) * U3[c * d3 + k] *
                   cg_racah(l1, i - l1, l2, j - l2, l3, k - l3);
          }
        }
        T[(a * d2 + b) * d3 + c] = acc;
      }
  double mre = 0, mim = 0;
  for (auto& z : T) {
    mre = std::fmax(mre, std::fabs(z.real()));
    mim = std::fmax(mim, std::fabs(z.imag()));
  }
  out.assign(T.size(), 0.0);
  double nrm = 0;
  for (size_t q = 0; q < T.size(); ++q) {
    out[q] = (mim > mre) ? T[q].imag() : T[q].real();
    nrm += out[q] * out[q];
  }
  nrm = std::sqrt(nrm);
  double sign = 0;
  for (size_t q = 0; q < out.size(); ++q) {
    out[q] /= nrm;
    if (sign == 0 && std::fabs(out[q]) > 1e-10) sign = out[q] > 0 ? 1.0 : -1.0;
  }
  for (auto& v : out) {
    v *= sign;
    if (std::fabs(v) < 1e-14) v = 0.0;
  }
}

// W[a][b][c] over S x S x S_out (S_out = S, or 1 for the last layer, which keeps
// only the scalar output 0e).
void fused_layer_tensor(int lmax, const float* theta_raw, std::vector<double>& W, int& n_in, int& n_out,
                        bool last) {
  const int S = (lmax + 1) * (lmax + 1);
  const int lm = lmax + 1;
  const int lo_max = last ? 0 : lmax;
  n_in = S;
  n_out = last ? 1 : S;
  W.assign((size_t)S * S * n_out, 0.0);
  auto pidx = [](int l) { return (l & 1) ? 1 : 0; };   // natural parity (-1)^l -> index
  for (int lo = 0; lo <= lo_max; ++lo) {
    int npaths = 0;
    for (int l1 = 0; l1 <= lmax; ++l1)
      for (int l2 = 0; l2 <= lmax; ++l2)
        if (lo >= std::abs(l1 - l2) && lo <= l1 + l2 && ((l1 + l2 + lo) % 2 == 0)) ++npaths;
    for (int l1 = 0; l1 <= lmax; ++l1)
      for (int l2 = 0; l2 <= lmax; ++l2) {
        if (!(lo >= std::abs(l1 - l2) && lo <= l1 + l2 && ((l1 + l2 + lo) % 2 == 0))) continue;
        // raw table [lo][po][l1][p1][l2], parity index 0 for +1, 1 for -1
        size_t idx = ((((size_t)lo * 2 + pidx(lo)) * lm + l1) * 2 + pidx(l1)) * lm + l2;
        double th = (double)theta_raw[idx] / std::sqrt((double)npaths);
        std::vector<double> Cc;
        coupling_real(l1, l2, lo, Cc);
        const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * lo + 1;
        for (int m1 = 0; m1 < d1; ++m1)
          for (int m2 = 0; m2 < d2; ++m2)
            for (int m3 = 0; m3 < d3; ++m3) {
              int a = l1 * l1 + m1, b = l2 * l2 + m2, c = lo * lo + m3;
              W[((size_t)a * S + b) * n_out + c] += th * Cc[(m1 * d2 + m2) * d3 + m3];
            }
      }
  }
}

// ---------------------------------------------------------------------------
// Models with more than two layers: features of the middle layers carry
// irreps (l, p) of either parity.  Layer L's outputs are the irreps (lo, po),
// lo <= l_max, produced by (l1, p1) x (l2, (-1)^l2) from its inputs that can
// still reach the scalar 0e in the remaining layers; the last layer keeps 0e
// only.  Irreps are ordered by l, then p = +1 before p = -1, each taking
// 2l + 1 consecutive components of the strided layout.
// ---------------------------------------------------------------------------
static void sort_unique(std::vector<Irrep>& v) {
  std::vector<Irrep> out;
  for (int l = 0; l <= 64; ++l)
    for (int p : {1, -1})
      for (const Irrep& x : v)
        if (x.l == l && x.p == p) {
          out.push_back(x);
          break;
        }
  v.swap(out);
}

static std::vector<Irrep> tp_outputs(const std::vector<Irrep>& in, int lmax) {
  std::vector<Irrep> out;
  for (const Irrep& a : in)
    for (int l2 = 0; l2 <= lmax; ++l2)
      for (int lo = std::abs(a.l - l2); lo <= std::min(a.l + l2, lmax); ++lo)
        out.push_back({lo, a.p * ((l2 & 1) ? -1 : 1)});
  sort_unique(out);
  return out;
}

static bool can_reach_scalar(const Irrep& ir, int steps, int lmax) {
  if (steps == 0) return ir.l == 0 && ir.p == 1;
  for (const Irrep& o : tp_outputs({ir}, lmax))
    if (can_reach_scalar(o, steps - 1, lmax)) return true;
  return false;
}

void layer_irreps(int lmax, int nl, std::vector<std::vector<Irrep>>& irs) {
  irs.clear();
  std::vector<Irrep> v0;
  for (int l = 0; l <= lmax; ++l) v0.push_back({l, (l & 1) ? -1 : 1});
  irs.push_back(v0);
  for (int L = 1; L <= nl; ++L) {
    std::vector<Irrep> keep;
    for (const Irrep& o : tp_outputs(irs.back(), lmax))
      if (can_reach_scalar(o, nl - L, lmax)) keep.push_back(o);
    irs.push_back(keep);
  }
}

int irreps_dim(const std::vector<Irrep>& v) {
  int d = 0;
  for (const Irrep& x : v) d += 2 * x.l + 1;
  return d;
}

// W[a][b][c] over dim(in) x S x dim(out) for the layer in -> out.
void layer_tensor(int lmax, const std::vector<Irrep>& in, const std::vector<Irrep>& out, const float* theta_raw,
                  std::vector<double>& W) {
  const int S = (lmax + 1) * (lmax + 1), lm = lmax + 1;
  const int din = irreps_dim(in), dout = irreps_dim(out);
  W.assign((size_t)din * S * dout, 0.0);
  auto pidx = [](int p) { return p == 1 ? 0 : 1; };
  std::vector<int> off_in, off_out;
  for (int o = 0, k = 0; k < (int)in.size(); o += 2 * in[k].l + 1, ++k) off_in.push_back(o);
  for (int o = 0, k = 0; k < (int)out.size(); o += 2 * out[k].l + 1, ++k) off_out.push_back(o);
  for (int ko = 0; ko < (int)out.size(); ++ko) {
    const int lo = out[ko].l, po = out[ko].p;
    int npaths = 0;
    for (const Irrep& a : in)
      for (int l2 = 0; l2 <= lmax; ++l2)
        if (lo >= std::abs(a.l - l2) && lo <= a.l + l2 && po == a.p * ((l2 & 1) ? -1 : 1)) ++npaths;
    for (int ki = 0; ki < (int)in.size(); ++ki) {
      const int l1 = in[ki].l, p1 = in[ki].p;
      for (int l2 = 0; l2 <= lmax; ++l2) {
        if (!(lo >= std::abs(l1 - l2) && lo <= l1 + l2 && po == p1 * ((l2 & 1) ? -1 : 1))) continue;
        const size_t idx = ((((size_t)lo * 2 + pidx(po)) * lm + l1) * 2 + pidx(p1)) * lm + l2;
        const double th = (double)theta_raw[idx] / std::sqrt((double)npaths);
        std::vector<double> Cc;
        coupling_real(l1, l2, lo, Cc);
        const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, d3 = 2 * lo + 1;
        for (int m1 = 0; m1 < d1; ++m1)
          for (int m2 = 0; m2 < d2; ++m2)
            for (int m3 = 0; m3 < d3; ++m3) {
              const int a = off_in[ki] + m1, b = l2 * l2 + m2, c = off_out[ko] + m3;
              W[((size_t)a * S + b) * dout + c] += th * Cc[(m1 * d2 + m2) * d3 + m3];
            }
      }
    }
  }
}

}  // namespace alg
