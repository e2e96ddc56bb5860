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
// Channel sums (the adjoint of Y, which is shared by all channels) are warp
// shuffles plus a fixed-order shared-memory combine: bitwise reproducible.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace alg {

template <typename T> __device__ __forceinline__ T to_act2(float v);
template <> __device__ __forceinline__ float to_act2<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 to_act2<bf16>(float v) { return __float2bfloat16_rn(v); }

template <int LMAX>
struct LOf {
  static __device__ __forceinline__ constexpr int l(int a) { return a < 1 ? 0 : (a < 4 ? 1 : (a < 9 ? 2 : 3)); }
};

// Sum v[0..S) over the block's C channel threads (C a power of two); the result
// for component b lands in `out[b]` (shared), valid after the call for every thread.
template <int S>
__device__ __forceinline__ void channel_sum(float (&v)[S], int C, float* red /*[4][S]*/, float* out /*[S]*/) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int width = C < 32 ? C : 32;
#pragma unroll
  for (int b = 0; b < S; ++b) {
    float x = v[b];
    for (int o = width >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu >> (32 - width), x, o);
    v[b] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < S; ++b) red[w * S + b] = v[b];
  }
  __syncthreads();
  const int nw = (C + 31) >> 5;
  for (int b = threadIdx.x; b < S; b += blockDim.x) {
    float s = 0.0f;
    for (int q = 0; q < nw; ++q) s += red[q * S + b];
    out[b] = s;
  }
  __syncthreads();
}

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
  for (int e = rb; e < re; ++e) {
    const float* w1 = io.W01 + (size_t)e * io.ld01 + nw + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = w1[l];
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
  for (int e = rb; e < re; ++e) {
    const float* w0 = io.W01 + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = w0[l];
    float s = 0.0f;
#pragma unroll
    for (int p = 0; p < S; ++p) s += wl[LOf<LMAX>::l(p)] * Y[p] * M0[p];
    xs[(size_t)e * io.ldxs + io.xs_off + u] = to_act2<T>(s);
  }
}

// ---------------------------------------------------------------------------
// forward, last layer NL: Gamma^NL and s^NL = sum_a clast[a] V^{NL-1}_a Gamma_a
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int NL>
__global__ void row_fwd_last_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  const float* wsrc = (NL == 1) ? io.W01 + nw : io.w2;
  const int ldw = (NL == 1) ? io.ld01 : io.ld2;
  float G[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G[b] = 0.0f;
  for (int e = rb; e < re; ++e) {
    const float* w = wsrc + (size_t)e * ldw + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = w[l];
#pragma unroll
    for (int b = 0; b < S; ++b) G[b] += wl[LOf<LMAX>::l(b)] * Y[b];
  }
  float* Gout = (NL == 1) ? io.G1 : io.G2;
#pragma unroll
  for (int b = 0; b < S; ++b) {
    G[b] *= tp.nu;
    Gout[((size_t)a * C + u) * S + b] = G[b];
  }
  float M[NL == 2 ? S * S : 1];
  if constexpr (NL == 2) {
    float G1[S];
#pragma unroll
    for (int b = 0; b < S; ++b) G1[b] = io.G1[((size_t)a * C + u) * S + b];
#pragma unroll
    for (int p = 0; p < S; ++p)
#pragma unroll
      for (int c = 0; c < S; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int b = 0; b < S; ++b) s += tp.W1[(p * S + b) * S + c] * G1[b];
        M[p * S + c] = s;
      }
  }
  float cg[S];
#pragma unroll
  for (int b = 0; b < S; ++b) cg[b] = tp.clast[b] * G[b];
  T* xs = reinterpret_cast<T*>(io.xs);
  for (int e = rb; e < re; ++e) {
    const float* w0 = io.W01 + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    float V[S];
#pragma unroll
    for (int p = 0; p < S; ++p) V[p] = w0[LOf<LMAX>::l(p)] * Y[p];
    float s = 0.0f;
    if constexpr (NL == 2) {
#pragma unroll
      for (int c = 0; c < S; ++c) {
        float v1 = 0.0f;
#pragma unroll
        for (int p = 0; p < S; ++p) v1 += V[p] * M[p * S + c];
        s += cg[c] * v1;
      }
    } else {
#pragma unroll
      for (int c = 0; c < S; ++c) s += cg[c] * V[c];
    }
    xs[(size_t)e * io.ldxs + io.xs_off + u] = to_act2<T>(s);
  }
}

// ---------------------------------------------------------------------------
// adjoint, last layer NL.  Given sbar^NL[e][u]:
//   Gammabar_b = sum_e sbar_e clast[b] V^{NL-1}_{e,b}       (per atom)
//   wbar^NL_{e,u,l} = nu sum_m Gammabar_(l,m) Y_{e,(l,m)}
//   Ybar_e[b] (+)= nu sum_u w^NL_{e,u,l(b)} Gammabar_{u,b}
// and for a one-layer model (V^{NL-1} = V^0 = w^0 Y) also
//   V0bar_b = sbar clast[b] Gamma_b;  wbar^0_{l} = sum_m V0bar Y;  Ybar += sum_u w^0 V0bar.
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int NL>
__global__ void row_bwd_last_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  __shared__ float red[4 * S];
  __shared__ float ysum[S];
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  const float* Gl = (NL == 1) ? io.G1 : io.G2;
  const float* sbar = (NL == 1) ? io.sbar1 : io.sbar2;
  const int lds = (NL == 1) ? io.ld_sbar1 : io.ld_sbar2;
  float G[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G[b] = Gl[((size_t)a * C + u) * S + b];
  float M[NL == 2 ? S * S : 1];
  if constexpr (NL == 2) {
    float G1[S];
#pragma unroll
    for (int b = 0; b < S; ++b) G1[b] = io.G1[((size_t)a * C + u) * S + b];
#pragma unroll
    for (int p = 0; p < S; ++p)
#pragma unroll
      for (int c = 0; c < S; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int b = 0; b < S; ++b) s += tp.W1[(p * S + b) * S + c] * G1[b];
        M[p * S + c] = s;
      }
  }
  T* wb01 = reinterpret_cast<T*>(io.wbar01);
  float Gb[S];
#pragma unroll
  for (int b = 0; b < S; ++b) Gb[b] = 0.0f;
  // pass 1
  for (int e = rb; e < re; ++e) {
    const float* w0 = io.W01 + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    const float sb = sbar[(size_t)e * lds + u];
    float w0l[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) w0l[l] = w0[l];
    float V[S];
#pragma unroll
    for (int p = 0; p < S; ++p) V[p] = w0l[LOf<LMAX>::l(p)] * Y[p];
    if constexpr (NL == 2) {
      float V1[S];
#pragma unroll
      for (int c = 0; c < S; ++c) {
        float v1 = 0.0f;
#pragma unroll
        for (int p = 0; p < S; ++p) v1 += V[p] * M[p * S + c];
        V1[c] = v1;
      }
#pragma unroll
      for (int b = 0; b < S; ++b) Gb[b] += sb * tp.clast[b] * V1[b];
    } else {
#pragma unroll
      for (int b = 0; b < S; ++b) Gb[b] += sb * tp.clast[b] * V[b];
      // V^0 adjoint: V0bar_b = sb clast[b] G_b
      float V0b[S];
#pragma unroll
      for (int b = 0; b < S; ++b) V0b[b] = sb * tp.clast[b] * G[b];
      float wl[LM];
#pragma unroll
      for (int l = 0; l < LM; ++l) wl[l] = 0.0f;
#pragma unroll
      for (int b = 0; b < S; ++b) wl[LOf<LMAX>::l(b)] += V0b[b] * Y[b];
#pragma unroll
      for (int l = 0; l < LM; ++l) wb01[(size_t)e * io.ld_wbar01 + u * LM + l] = to_act2<T>(wl[l]);
      float yc[S];
#pragma unroll
      for (int b = 0; b < S; ++b) yc[b] = w0l[LOf<LMAX>::l(b)] * V0b[b];
      channel_sum<S>(yc, C, red, ysum);
      for (int b = u; b < S; b += C) io.Ybar[(size_t)e * S + b] = ysum[b];
    }
  }
  // pass 2
  T* wbL = (NL == 1) ? wb01 + nw : reinterpret_cast<T*>(io.wbar2);
  const int ldwb = (NL == 1) ? io.ld_wbar01 : io.ld_wbar2;
  const float* wsrc = (NL == 1) ? io.W01 + nw : io.w2;
  const int ldw = (NL == 1) ? io.ld01 : io.ld2;
  for (int e = rb; e < re; ++e) {
    const float* Y = io.Y + (size_t)e * S;
    const float* w = wsrc + (size_t)e * ldw + u * LM;
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = 0.0f;
#pragma unroll
    for (int b = 0; b < S; ++b) wl[LOf<LMAX>::l(b)] += Gb[b] * Y[b];
#pragma unroll
    for (int l = 0; l < LM; ++l) wbL[(size_t)e * ldwb + u * LM + l] = to_act2<T>(tp.nu * wl[l]);
    float yc[S];
#pragma unroll
    for (int b = 0; b < S; ++b) yc[b] = tp.nu * w[LOf<LMAX>::l(b)] * Gb[b];
    channel_sum<S>(yc, C, red, ysum);
    for (int b = u; b < S; b += C) {
      if (NL == 1) io.Ybar[(size_t)e * S + b] += ysum[b];
      else io.Ybar[(size_t)e * S + b] = ysum[b];
    }
  }
}

// ---------------------------------------------------------------------------
// adjoint, layer 1 of a two-layer model.  Given sbar^1, sbar^2:
//   V1bar_c = clast[c] sbar^2 Gamma^2_c + [c == 0] sbar^1
//   Gamma1bar_b = sum_e sum_{a,c} W1[a][b][c] V0_{e,a} V1bar_{e,c}     (per atom)
//   V0bar_a = sum_c M1[a][c] V1bar_c,  M1 = W1 . Gamma^1
//   wbar^0_l = sum_m V0bar_(l,m) Y_(l,m);  wbar^1_l = nu sum_m Gamma1bar_(l,m) Y_(l,m)
//   Ybar_e[a] += sum_u (w^0_{l(a)} V0bar_a + nu w^1_{l(a)} Gamma1bar_a)
// ---------------------------------------------------------------------------
template <typename T, int LMAX>
__global__ void row_bwd_mid_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  __shared__ float red[4 * S];
  __shared__ float ysum[S];
  const int a = blockIdx.x, u = threadIdx.x, C = io.C;
  const int rb = io.row_ptr[io.a0 + a] - io.e0, re = io.row_ptr[io.a0 + a + 1] - io.e0;
  const int nw = C * LM;
  float G2[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G2[b] = tp.clast[b] * io.G2[((size_t)a * C + u) * S + b];
  float P[S * S];
#pragma unroll
  for (int q = 0; q < S * S; ++q) P[q] = 0.0f;
  for (int e = rb; e < re; ++e) {
    const float* w0 = io.W01 + (size_t)e * io.ld01 + u * LM;
    const float* Y = io.Y + (size_t)e * S;
    const float sb1 = io.sbar1[(size_t)e * io.ld_sbar1 + u];
    const float sb2 = io.sbar2[(size_t)e * io.ld_sbar2 + u];
    float V0[S], V1b[S];
#pragma unroll
    for (int p = 0; p < S; ++p) V0[p] = w0[LOf<LMAX>::l(p)] * Y[p];
#pragma unroll
    for (int c = 0; c < S; ++c) V1b[c] = sb2 * G2[c] + (c == 0 ? sb1 : 0.0f);
#pragma unroll
    for (int p = 0; p < S; ++p)
#pragma unroll
      for (int c = 0; c < S; ++c) P[p * S + c] += V0[p] * V1b[c];
  }
  float G1b[S];
#pragma unroll
  for (int b = 0; b < S; ++b) {
    float s = 0.0f;
#pragma unroll
    for (int p = 0; p < S; ++p)
#pragma unroll
      for (int c = 0; c < S; ++c) s += tp.W1[(p * S + b) * S + c] * P[p * S + c];
    G1b[b] = s;
  }
  float G1[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G1[b] = io.G1[((size_t)a * C + u) * S + b];
  float M[S * S];
#pragma unroll
  for (int p = 0; p < S; ++p)
#pragma unroll
    for (int c = 0; c < S; ++c) {
      float s = 0.0f;
#pragma unroll
      for (int b = 0; b < S; ++b) s += tp.W1[(p * S + b) * S + c] * G1[b];
      M[p * S + c] = s;
    }
  T* wb = reinterpret_cast<T*>(io.wbar01);
  for (int e = rb; e < re; ++e) {
    const float* w0 = io.W01 + (size_t)e * io.ld01 + u * LM;
    const float* w1 = w0 + nw;
    const float* Y = io.Y + (size_t)e * S;
    const float sb1 = io.sbar1[(size_t)e * io.ld_sbar1 + u];
    const float sb2 = io.sbar2[(size_t)e * io.ld_sbar2 + u];
    float V1b[S];
#pragma unroll
    for (int c = 0; c < S; ++c) V1b[c] = sb2 * G2[c] + (c == 0 ? sb1 : 0.0f);
    float V0b[S];
#pragma unroll
    for (int p = 0; p < S; ++p) {
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < S; ++c) s += M[p * S + c] * V1b[c];
      V0b[p] = s;
    }
    float w0l[LM], w1l[LM], g0[LM], g1[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) { w0l[l] = w0[l]; w1l[l] = w1[l]; g0[l] = 0.0f; g1[l] = 0.0f; }
#pragma unroll
    for (int b = 0; b < S; ++b) {
      g0[LOf<LMAX>::l(b)] += V0b[b] * Y[b];
      g1[LOf<LMAX>::l(b)] += G1b[b] * Y[b];
    }
#pragma unroll
    for (int l = 0; l < LM; ++l) {
      wb[(size_t)e * io.ld_wbar01 + u * LM + l] = to_act2<T>(g0[l]);
      wb[(size_t)e * io.ld_wbar01 + nw + u * LM + l] = to_act2<T>(tp.nu * g1[l]);
    }
    float yc[S];
#pragma unroll
    for (int b = 0; b < S; ++b) yc[b] = w0l[LOf<LMAX>::l(b)] * V0b[b] + tp.nu * w1l[LOf<LMAX>::l(b)] * G1b[b];
    channel_sum<S>(yc, C, red, ysum);
    for (int b = u; b < S; b += C) io.Ybar[(size_t)e * S + b] += ysum[b];
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
  if (layer < nl) {
    if (lmax == 1) row_bwd_mid_kernel<T, 1><<<grid, block, 0, st>>>(io, tp);
    else row_bwd_mid_kernel<T, 2><<<grid, block, 0, st>>>(io, tp);
  } else if (nl == 1) {
    if (lmax == 1) row_bwd_last_kernel<T, 1, 1><<<grid, block, 0, st>>>(io, tp);
    else row_bwd_last_kernel<T, 2, 1><<<grid, block, 0, st>>>(io, tp);
  } else {
    if (lmax == 1) row_bwd_last_kernel<T, 1, 2><<<grid, block, 0, st>>>(io, tp);
    else row_bwd_last_kernel<T, 2, 2><<<grid, block, 0, st>>>(io, tp);
  }
}

template void row_fwd<float>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_fwd<bf16>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_bwd<float>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_bwd<bf16>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);

}  // namespace alg
