// Row (per-centre-atom) kernels: the environment embedding and the tensor
// product of Eq. 1, forward and adjoint.
//
// Eq. 1 (bilinearity): V^{ij,L} = V^{ij,L-1} (x) Gamma^{i,L},
//   Gamma^{i,L}_{u,(l,m)} = nu * sum_{k in N(i)} w^{ik,L}_{u,l} Y_{lm}(r_ik),
// so each product needs one environment per centre atom i.  A block owns one
// centre atom and its whole CSR row (all edges (i, j)); thread u owns
// channel u (the tensor product is channel-wise: the u index is shared).  The
// per-atom sums over the row are register accumulations -- deterministic, no
// atomics -- and per-edge results are written in the same kernel.
//
// Tensor product with the strided layout and fused path weights (Sec.
// "Optimized tensor product"): V^L_c = sum_{a,b} W[a][b][c] V^{L-1}_a Gamma_b.
// Per atom the kernel first contracts W with Gamma (M[a][c] = sum_b W[a][b][c]
// Gamma_b, the cheap order: once per atom), then each edge costs S x S FMAs.
// The last layer keeps only the scalar output; its W[a][b][0] is diagonal
// (w3j(l,l,0) pairs m1 = m2), so s = sum_a clast[a] V_a Gamma_a (the paper's
// removal of the redundant dimension).
//
// Channel sums (the adjoint of Y, which is shared by all channels) go through
// shared memory a few edges at a time, in a fixed order: bitwise reproducible.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace alg {

__device__ __forceinline__ float ld_act(const float* p) { return *p; }
__device__ __forceinline__ float ld_act(const bf16* p) { return __bfloat162float(*p); }

template <typename T> __device__ __forceinline__ T to_act2(float v);
template <> __device__ __forceinline__ float to_act2<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 to_act2<bf16>(float v) { return __float2bfloat16_rn(v); }

template <int LMAX>
struct LOf {
  static __device__ __forceinline__ constexpr int l(int a) { return a < 1 ? 0 : (a < 4 ? 1 : (a < 9 ? 2 : 3)); }
};

// ---------------------------------------------------------------------------
// forward, layer 1 of a two-layer model: Gamma^1 and s^1 = V^1_{0e}
// ---------------------------------------------------------------------------
template <typename T, int LMAX>
__global__ void row_fwd_mid_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  float G[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G[b] = 0.0f;
#pragma unroll 4
  for (int e = rb; e < re; ++e) {
    const T* w1 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + nw + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = ld_act(w1 + l);
#pragma unroll
    for (int b = 0; b < S; ++b) G[b] += wl[LOf<LMAX>::l(b)] * Y[b];
  }
#pragma unroll
  for (int b = 0; b < S; ++b) {
    G[b] *= tp.nu;
    io.G1[((size_t)a * C + u) * S + b] = G[b];
  }
  // only the scalar output c = 0 is needed here: M0[a'] = sum_b W[a'][b][0] G_b
  float M0[S];
#pragma unroll
  for (int p = 0; p < S; ++p) {
    float s = 0.0f;
#pragma unroll
    for (int b = 0; b < S; ++b) s += tp.W1[(p * S + b) * S + 0] * G[b];
    M0[p] = s;
  }
  T* xs = reinterpret_cast<T*>(io.xs);
#pragma unroll 4
  for (int e = rb; e < re; ++e) {
    const T* w0 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = ld_act(w0 + l);
    float s = 0.0f;
#pragma unroll
    for (int p = 0; p < S; ++p) s += wl[LOf<LMAX>::l(p)] * Y[p] * M0[p];
    xs[(size_t)e * io.ldxs + io.xs_off + u] = to_act2<T>(s);
  }
}

// ---------------------------------------------------------------------------
// Factorised products.  With the scalar-only last layer, every product that
// involves V^1 = V^0 . M^1 (M^1_{ac} = sum_b W1[a][b][c] Gamma^1_b) collapses
// to per-atom vectors, so each edge costs O(S) per channel:
//   s^2            = sum_a V^0_a T2_a,           T2_a = sum_{b,c} W1[a][b][c] Gamma^1_b cg2_c
//   Gamma^2bar_b   = clast_b sum_a M^1_{ab} Q2_a,  Q2_a = sum_e sbar^2_e V^0_{e,a}
//   V^0bar_a       = sbar^2 T2_a + sbar^1 T1_a,  T1_a = M^1_{a0}
//   Gamma^1bar_b   = sum_{a,c} W1[a][b][c] (cg2_c Q2_a + [c = 0] Q1_a),  Q1_a = sum_e sbar^1_e V^0_{e,a}
// with cg2_c = clast_c Gamma^2_c.  (The general S x S per-edge products are
// what these reduce to; the reduction is exact, only the summation order
// changes.)
// ---------------------------------------------------------------------------

// T2[a] = sum_{b,c} W1[a][b][c] G1[b] cg[c]
template <int S>
__device__ __forceinline__ void make_T2(const TPConst& tp, const float (&G1)[S], const float (&cg)[S], float (&T2)[S]) {
#pragma unroll
  for (int p = 0; p < S; ++p) {
    float t = 0.0f;
#pragma unroll
    for (int b = 0; b < S; ++b) {
      float r = 0.0f;
#pragma unroll
      for (int c = 0; c < S; ++c) r += tp.W1[(p * S + b) * S + c] * cg[c];
      t += G1[b] * r;
    }
    T2[p] = t;
  }
}

// Channel sums of per-edge S-vectors, EB edges at a time, through shared
// memory laid out [EB][S][C+1] (conflict-free), fixed summation order.
template <int S>
struct YSum {
  float* red;
  int C;
  __device__ __forceinline__ void put(int k, const float (&v)[S]) const {
#pragma unroll
    for (int b = 0; b < S; ++b) red[(k * S + b) * (C + 1) + threadIdx.x] = v[b];
  }
  // writes (accumulate = false) or adds the sums into Ybar rows e0 .. e0+nk-1
  __device__ __forceinline__ void flush(float* Ybar, int e0, int nk, bool accumulate) const {
    __syncthreads();
    for (int t = threadIdx.x; t < nk * S; t += C) {
      const float* row = red + t * (C + 1);
      float s = 0.0f;
      for (int q = 0; q < C; ++q) s += row[q];
      const int k = t / S, b = t - k * S;
      float* y = Ybar + (size_t)(e0 + k) * S + b;
      *y = accumulate ? *y + s : s;
    }
    __syncthreads();
  }
};

constexpr int kEB = 4;   // edges per channel-sum batch

template <int S>
__host__ __device__ constexpr size_t ysum_smem(int C) {
  return (size_t)kEB * S * (C + 1) * sizeof(float);
}

// ---------------------------------------------------------------------------
// forward, last layer NL: Gamma^NL and s^NL
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int NL>
__global__ void row_fwd_last_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  const T* wsrc = (NL == 1) ? reinterpret_cast<const T*>(io.W01) + nw : reinterpret_cast<const T*>(io.w2);
  const int ldw = (NL == 1) ? io.ld01 : io.ld2;
  float G[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G[b] = 0.0f;
#pragma unroll 4
  for (int e = rb; e < re; ++e) {
    const T* w = wsrc + (size_t)e * ldw + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = ld_act(w + l);
#pragma unroll
    for (int b = 0; b < S; ++b) G[b] += wl[LOf<LMAX>::l(b)] * Y[b];
  }
  float* Gout = (NL == 1) ? io.G1 : io.G2;
  float cg[S];
#pragma unroll
  for (int b = 0; b < S; ++b) {
    G[b] *= tp.nu;
    Gout[((size_t)a * C + u) * S + b] = G[b];
    cg[b] = tp.clast[b] * G[b];
  }
  float Tv[S];
  if constexpr (NL == 2) {
    float G1[S];
#pragma unroll
    for (int b = 0; b < S; ++b) G1[b] = io.G1[((size_t)a * C + u) * S + b];
    make_T2<S>(tp, G1, cg, Tv);
  } else {
#pragma unroll
    for (int b = 0; b < S; ++b) Tv[b] = cg[b];
  }
  T* xs = reinterpret_cast<T*>(io.xs);
#pragma unroll 4
  for (int e = rb; e < re; ++e) {
    const T* w0 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = ld_act(w0 + l);
    float s = 0.0f;
#pragma unroll
    for (int p = 0; p < S; ++p) s += wl[LOf<LMAX>::l(p)] * Y[p] * Tv[p];
    xs[(size_t)e * io.ldxs + io.xs_off + u] = to_act2<T>(s);
  }
}

// ---------------------------------------------------------------------------
// adjoint, last layer NL.  Given sbar^NL[e][u]:
//   NL = 2:  Gamma^2bar = clast . (M^1^T Q2);  wbar^2 and Ybar (=) from Gamma^2bar
//   NL = 1:  Gamma^1bar_b = clast_b sum_e sbar_e V^0_{e,b};  V^0bar = sbar clast Gamma^1;
//            wbar^0, wbar^1 and Ybar (=) in one pass
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int NL>
__global__ void row_bwd_last_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  extern __shared__ float red_dyn[];
  const YSum<S> ys{red_dyn, io.C};
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  const float* Gl = (NL == 1) ? io.G1 : io.G2;
  const float* sbar = (NL == 1) ? io.sbar1 : io.sbar2;
  const int lds = (NL == 1) ? io.ld_sbar1 : io.ld_sbar2;
  float G[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G[b] = Gl[((size_t)a * C + u) * S + b];
  // pass 1: Q[a] = sum_e sbar_e V^0_{e,a}
  float Q[S];
#pragma unroll
  for (int b = 0; b < S; ++b) Q[b] = 0.0f;
#pragma unroll 4
  for (int e = rb; e < re; ++e) {
    const T* w0 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    const float sb = sbar[(size_t)e * lds + u];
    float w0l[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) w0l[l] = ld_act(w0 + l);
#pragma unroll
    for (int b = 0; b < S; ++b) Q[b] += sb * w0l[LOf<LMAX>::l(b)] * Y[b];
  }
  float Gb[S];
  if constexpr (NL == 2) {
    float G1[S];
#pragma unroll
    for (int b = 0; b < S; ++b) {
      G1[b] = io.G1[((size_t)a * C + u) * S + b];
      Gb[b] = 0.0f;
    }
#pragma unroll
    for (int p = 0; p < S; ++p)
#pragma unroll
      for (int bp = 0; bp < S; ++bp) {
        const float gq = G1[bp] * Q[p];
#pragma unroll
        for (int b = 0; b < S; ++b) Gb[b] += tp.W1[(p * S + bp) * S + b] * gq;
      }
#pragma unroll
    for (int b = 0; b < S; ++b) Gb[b] *= tp.clast[b];
  } else {
#pragma unroll
    for (int b = 0; b < S; ++b) Gb[b] = tp.clast[b] * Q[b];
  }
  // pass 2
  T* wb01 = reinterpret_cast<T*>(io.wbar01);
  T* wbL = (NL == 1) ? wb01 + nw : reinterpret_cast<T*>(io.wbar2);
  const int ldwb = (NL == 1) ? io.ld_wbar01 : io.ld_wbar2;
  const T* wsrc = (NL == 1) ? reinterpret_cast<const T*>(io.W01) + nw : reinterpret_cast<const T*>(io.w2);
  const int ldw = (NL == 1) ? io.ld01 : io.ld2;
  for (int eg = rb; eg < re; eg += kEB) {
    const int nk = min(kEB, re - eg);
    for (int k = 0; k < nk; ++k) {
      const int e = eg + k;
      const float* Y = io.Y + (size_t)e * S;
      const T* w = wsrc + (size_t)e * ldw + u * LM;
      float wl[LM], gl[LM];
#pragma unroll
      for (int l = 0; l < LM; ++l) { wl[l] = ld_act(w + l); gl[l] = 0.0f; }
#pragma unroll
      for (int b = 0; b < S; ++b) gl[LOf<LMAX>::l(b)] += Gb[b] * Y[b];
#pragma unroll
      for (int l = 0; l < LM; ++l) wbL[(size_t)e * ldwb + u * LM + l] = to_act2<T>(tp.nu * gl[l]);
      float yc[S];
#pragma unroll
      for (int b = 0; b < S; ++b) yc[b] = tp.nu * wl[LOf<LMAX>::l(b)] * Gb[b];
      if constexpr (NL == 1) {
        const float sb = sbar[(size_t)e * lds + u];
        const T* w0 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + u * LM;
        float w0l[LM], g0[LM];
#pragma unroll
        for (int l = 0; l < LM; ++l) { w0l[l] = ld_act(w0 + l); g0[l] = 0.0f; }
#pragma unroll
        for (int b = 0; b < S; ++b) {
          const float v0b = sb * tp.clast[b] * G[b];
          g0[LOf<LMAX>::l(b)] += v0b * Y[b];
          yc[b] += w0l[LOf<LMAX>::l(b)] * v0b;
        }
#pragma unroll
        for (int l = 0; l < LM; ++l) wb01[(size_t)e * io.ld_wbar01 + u * LM + l] = to_act2<T>(g0[l]);
      }
      ys.put(k, yc);
    }
    ys.flush(io.Ybar, eg, nk, false);
  }
}

// ---------------------------------------------------------------------------
// adjoint, layer 1 of a two-layer model (factorised, see above):
//   pass 1: Q1 = sum_e sbar^1 V^0, Q2 = sum_e sbar^2 V^0
//   per atom: T1, T2, Gamma^1bar
//   pass 2: V^0bar = sbar^2 T2 + sbar^1 T1;  wbar^0_l = sum_m V^0bar Y;
//           wbar^1_l = nu sum_m Gamma^1bar Y;  Ybar += sum_u (w^0 V^0bar + nu w^1 Gamma^1bar)
// ---------------------------------------------------------------------------
template <typename T, int LMAX>
__global__ void row_bwd_mid_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  extern __shared__ float red_dyn[];
  const YSum<S> ys{red_dyn, io.C};
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  float Q1[S], Q2[S];
#pragma unroll
  for (int b = 0; b < S; ++b) { Q1[b] = 0.0f; Q2[b] = 0.0f; }
#pragma unroll 4
  for (int e = rb; e < re; ++e) {
    const T* w0 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    const float sb1 = io.sbar1[(size_t)e * io.ld_sbar1 + u];
    const float sb2 = io.sbar2[(size_t)e * io.ld_sbar2 + u];
    float w0l[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) w0l[l] = ld_act(w0 + l);
#pragma unroll
    for (int p = 0; p < S; ++p) {
      const float v0 = w0l[LOf<LMAX>::l(p)] * Y[p];
      Q1[p] += sb1 * v0;
      Q2[p] += sb2 * v0;
    }
  }
  float G1[S], cg2[S], T1[S], T2[S], G1b[S];
#pragma unroll
  for (int b = 0; b < S; ++b) {
    G1[b] = io.G1[((size_t)a * C + u) * S + b];
    cg2[b] = tp.clast[b] * io.G2[((size_t)a * C + u) * S + b];
    T1[b] = 0.0f; T2[b] = 0.0f; G1b[b] = 0.0f;
  }
#pragma unroll
  for (int p = 0; p < S; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) {
      float r = 0.0f;
#pragma unroll
      for (int c = 0; c < S; ++c) r += tp.W1[(p * S + b) * S + c] * cg2[c];
      const float w0c = tp.W1[(p * S + b) * S + 0];
      T2[p] += G1[b] * r;
      T1[p] += w0c * G1[b];
      G1b[b] += Q2[p] * r + Q1[p] * w0c;
    }
  T* wb = reinterpret_cast<T*>(io.wbar01);
  for (int eg = rb; eg < re; eg += kEB) {
    const int nk = min(kEB, re - eg);
    for (int k = 0; k < nk; ++k) {
      const int e = eg + k;
      const T* w0 = reinterpret_cast<const T*>(io.W01) + (size_t)e * io.ld01 + u * LM;
      const T* w1 = w0 + nw;
      const float* Y = io.Y + (size_t)e * S;
      const float sb1 = io.sbar1[(size_t)e * io.ld_sbar1 + u];
      const float sb2 = io.sbar2[(size_t)e * io.ld_sbar2 + u];
      float w0l[LM], w1l[LM], g0[LM], g1[LM];
#pragma unroll
      for (int l = 0; l < LM; ++l) { w0l[l] = ld_act(w0 + l); w1l[l] = ld_act(w1 + l); g0[l] = 0.0f; g1[l] = 0.0f; }
      float yc[S];
#pragma unroll
      for (int b = 0; b < S; ++b) {
        const float v0b = sb2 * T2[b] + sb1 * T1[b];
        g0[LOf<LMAX>::l(b)] += v0b * Y[b];
        g1[LOf<LMAX>::l(b)] += G1b[b] * Y[b];
        yc[b] = w0l[LOf<LMAX>::l(b)] * v0b + tp.nu * w1l[LOf<LMAX>::l(b)] * G1b[b];
      }
#pragma unroll
      for (int l = 0; l < LM; ++l) {
        wb[(size_t)e * io.ld_wbar01 + u * LM + l] = to_act2<T>(g0[l]);
        wb[(size_t)e * io.ld_wbar01 + nw + u * LM + l] = to_act2<T>(tp.nu * g1[l]);
      }
      ys.put(k, yc);
    }
    ys.flush(io.Ybar, eg, nk, true);
  }
}

// ---------------------------------------------------------------------------
template <typename T>
void row_fwd(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st) {
  if (io.na <= 0) return;
  dim3 grid(io.na), block(io.C);
  if (layer < nl) {
    if (lmax == 1) row_fwd_mid_kernel<T, 1><<<grid, block, 0, st>>>(io, tp);
    else row_fwd_mid_kernel<T, 2><<<grid, block, 0, st>>>(io, tp);
  } else if (nl == 1) {
    if (lmax == 1) row_fwd_last_kernel<T, 1, 1><<<grid, block, 0, st>>>(io, tp);
    else row_fwd_last_kernel<T, 2, 1><<<grid, block, 0, st>>>(io, tp);
  } else {
    if (lmax == 1) row_fwd_last_kernel<T, 1, 2><<<grid, block, 0, st>>>(io, tp);
    else row_fwd_last_kernel<T, 2, 2><<<grid, block, 0, st>>>(io, tp);
  }
}

template <typename T>
void row_bwd(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st) {
  if (io.na <= 0) return;
  dim3 grid(io.na), block(io.C);
  const size_t sm1 = ysum_smem<4>(io.C), sm2 = ysum_smem<9>(io.C);
  if (layer < nl) {
    if (lmax == 1) row_bwd_mid_kernel<T, 1><<<grid, block, sm1, st>>>(io, tp);
    else row_bwd_mid_kernel<T, 2><<<grid, block, sm2, st>>>(io, tp);
  } else if (nl == 1) {
    if (lmax == 1) row_bwd_last_kernel<T, 1, 1><<<grid, block, sm1, st>>>(io, tp);
    else row_bwd_last_kernel<T, 2, 1><<<grid, block, sm2, st>>>(io, tp);
  } else {
    if (lmax == 1) row_bwd_last_kernel<T, 1, 2><<<grid, block, sm1, st>>>(io, tp);
    else row_bwd_last_kernel<T, 2, 2><<<grid, block, sm2, st>>>(io, tp);
  }
}

template void row_fwd<float>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_fwd<bf16>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_bwd<float>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_bwd<bf16>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);

}  // namespace alg
