// Row (per-centre-atom) kernels: the environment embedding and the tensor
// product of Eq. 1, forward and adjoint.
//
// Eq. 1 (bilinearity): V^{ij,L} = V^{ij,L-1} (x) Gamma^{i,L},
//   Gamma^{i,L}_{u,(l,m)} = nu * sum_{k in N(i)} w^{ik,L}_{u,l} Y_{lm}(r_ik),
// so each product needs one environment per centre atom i.  One warp owns one
// centre atom and its whole CSR row (all edges (i, j)); lane t owns the CPL
// consecutive channels [CPL t, CPL t + CPL) (the tensor product is
// channel-wise: the u index is shared).  The per-atom sums over the row are
// register accumulations -- deterministic, no atomics -- and per-edge results
// are written in the same kernel.  A lane's per-edge weights (CPL (l_max+1)
// values) are one vector load; the row's Y values are staged once per segment
// in shared memory and read back as 16-byte vectors by every lane.
//
// Tensor product with the strided layout and fused path weights (Sec.
// "Optimized tensor product"): V^L_c = sum_{a,b} W[a][b][c] V^{L-1}_a Gamma_b.
// Per atom the kernel contracts W with Gamma once (M[a][c] = sum_b W[a][b][c]
// Gamma_b, the cheap order), then each edge costs O(S) per channel.  The
// per-atom contractions visit only the entries the coupling pattern allows
// (83 of 729 for l_max = 2; `tp_nonzero`), resolved at compile time.  The last
// layer keeps only the scalar output; its W[a][b][0] is diagonal (w3j(l,l,0)
// pairs m1 = m2), so s = sum_a clast[a] V_a Gamma_a (the paper's removal of the
// redundant dimension).
//
// Channel sums (the adjoint of Y, which is shared by all channels) are warp
// reductions with a fixed shuffle pattern: bitwise reproducible.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace alg {

namespace {

constexpr int kRowWarps = 4;   // atoms (warps) per block
constexpr int kYSeg = 64;      // edges per staged segment of Y

// A lane's channels are processed in pairs (2p, 2p + 1) with the packed fp32
// operations of sm_100 and later (one FFMA2 / FMUL2 for two channels); each
// half is an ordinary IEEE fp32 fma / multiply.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

template <int LMAX>
__device__ __forceinline__ constexpr int lof(int a) { return a < 1 ? 0 : (a < 4 ? 1 : (a < 9 ? 2 : 3)); }

// ---- vector access to a lane's span of N consecutive elements ------------
// The span starts at a multiple of its own byte size inside a 16-byte aligned
// row, so it is aligned to the largest power of two (<= 16) dividing that size.
template <int NB>
struct SpanAlign {
  static constexpr int v = (NB % 16 == 0) ? 16 : (NB % 8 == 0) ? 8 : 4;
  static_assert(NB % 4 == 0, "a lane span must be a whole number of 32-bit words");
};

template <int NB>
__device__ __forceinline__ void ld_words(const void* p, uint32_t (&w)[NB / 4]) {
  constexpr int AL = SpanAlign<NB>::v;
  if constexpr (AL == 16) {
#pragma unroll
    for (int i = 0; i < NB / 16; ++i) {
      const uint4 x = reinterpret_cast<const uint4*>(p)[i];
      w[4 * i] = x.x; w[4 * i + 1] = x.y; w[4 * i + 2] = x.z; w[4 * i + 3] = x.w;
    }
  } else if constexpr (AL == 8) {
#pragma unroll
    for (int i = 0; i < NB / 8; ++i) {
      const uint2 x = reinterpret_cast<const uint2*>(p)[i];
      w[2 * i] = x.x; w[2 * i + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NB / 4; ++i) w[i] = reinterpret_cast<const uint32_t*>(p)[i];
  }
}

template <int NB>
__device__ __forceinline__ void st_words(void* p, const uint32_t (&w)[NB / 4]) {
  constexpr int AL = SpanAlign<NB>::v;
  if constexpr (AL == 16) {
#pragma unroll
    for (int i = 0; i < NB / 16; ++i)
      reinterpret_cast<uint4*>(p)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  } else if constexpr (AL == 8) {
#pragma unroll
    for (int i = 0; i < NB / 8; ++i) reinterpret_cast<uint2*>(p)[i] = make_uint2(w[2 * i], w[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < NB / 4; ++i) reinterpret_cast<uint32_t*>(p)[i] = w[i];
  }
}

// bf16 -> float is exact: the bf16 bits are the upper half of the float.
template <typename T, int N>
__device__ __forceinline__ void unpack_span(const uint32_t (&w)[N * sizeof(T) / 4], float (&o)[N]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < N; ++k) o[k] = __uint_as_float(w[k]);
  } else {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
}

template <typename T, int N>
__device__ __forceinline__ void ld_span(const T* p, float (&o)[N]) {
  constexpr int NB = N * (int)sizeof(T);
  uint32_t w[NB / 4];
  ld_words<NB>(p, w);
  unpack_span<T, N>(w, o);
}

template <typename T, int N>
__device__ __forceinline__ void st_span(T* p, const float (&v)[N]) {
  constexpr int NB = N * (int)sizeof(T);
  uint32_t w[NB / 4];
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = __float_as_uint(v[k]);
  } else {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
      w[k] = *reinterpret_cast<uint32_t*>(&h);
    }
  }
  st_words<NB>(p, w);
}

template <typename T> __device__ __forceinline__ T to_act2(float v);
template <> __device__ __forceinline__ float to_act2<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 to_act2<bf16>(float v) { return __float2bfloat16_rn(v); }

// ---- Y staging: the row segment's Y values, padded to 16-byte records -----
template <int S>
struct YStage {
  static constexpr int P = (S + 3) & ~3;
  float* ys;   // this warp's [kYSeg][P]
  __device__ __forceinline__ void load(const float* Y, int e0, int cnt, int lane) const {
    __syncwarp();
    const float* src = Y + (size_t)e0 * S;
    for (int t = lane; t < cnt * S; t += 32) {
      const int k = t / S, b = t - k * S;
      ys[k * P + b] = src[t];
    }
    __syncwarp();
  }
  __device__ __forceinline__ void get(int k, float (&y)[S]) const {
    float v[P];
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
      const float4 x = reinterpret_cast<const float4*>(ys + k * P)[q];
      v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
#pragma unroll
    for (int b = 0; b < S; ++b) y[b] = v[b];
  }
};

// ---- channel sums of an S-vector over the warp (fixed pattern) ------------
// Reduce-scatter: after the exchanges at distance 16, 8 (and 4 for eight
// values) each lane holds the sum of one value index over the lanes that
// differ in those bits; the remaining distances complete the sum.  Writes
// the S sums into ybar[0..S).
__device__ __forceinline__ float rs_step(float lo, float hi, bool upper, int dist) {
  const float send = upper ? lo : hi;
  const float keep = upper ? hi : lo;
  return keep + __shfl_xor_sync(0xffffffffu, send, dist);
}

template <int S>
__device__ __forceinline__ void warp_channel_sum(const float (&v)[S], int lane, float* ybar) {
  if constexpr (S == 9) {
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = rs_step(v[i], v[i + 4], lane & 16, 16);
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = rs_step(a[i], a[i + 2], lane & 8, 8);
    float c = rs_step(b[0], b[1], lane & 4, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    float t = v[8];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
    if ((lane & 3) == 0) ybar[(lane >> 2) & 7] = c;
    if (lane == 1) ybar[8] = t;
  } else {
    static_assert(S == 4, "l_max 1 or 2");
    float a[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) a[i] = rs_step(v[i], v[i + 2], lane & 16, 16);
    float c = rs_step(a[0], a[1], lane & 8, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    if ((lane & 7) == 0) ybar[(lane >> 3) & 3] = c;
  }
}

struct RowCtx {
  int a, lane, u0, rb, re;
  bool act;
};

template <int CPL>
__device__ __forceinline__ bool row_ctx(const RowIO& io, RowCtx& r) {
  const int warp = threadIdx.x >> 5;
  r.lane = threadIdx.x & 31;
  r.a = blockIdx.x * kRowWarps + warp;
  if (r.a >= io.na) return false;
  r.u0 = CPL * r.lane;
  r.act = r.u0 < io.C;
  r.rb = io.row_ptr[io.a0 + r.a] - io.e0;
  r.re = io.row_ptr[io.a0 + r.a + 1] - io.e0;
  return true;
}

// per-atom [C][S] float arrays: lane's CPL x S block
template <int CPL, int S>
__device__ __forceinline__ void ld_atom(const float* base, const RowIO& io, const RowCtx& r, float (&o)[CPL][S]) {
  float t[CPL * S];
  if (r.act) ld_span<float, CPL * S>(base + ((size_t)r.a * io.C + r.u0) * S, t);
  else {
#pragma unroll
    for (int q = 0; q < CPL * S; ++q) t[q] = 0.0f;
  }
#pragma unroll
  for (int j = 0; j < CPL; ++j)
#pragma unroll
    for (int b = 0; b < S; ++b) o[j][b] = t[j * S + b];
}

template <int CPL, int S>
__device__ __forceinline__ void st_atom(float* base, const RowIO& io, const RowCtx& r, const float (&v)[CPL][S]) {
  if (!r.act) return;
  float t[CPL * S];
#pragma unroll
  for (int j = 0; j < CPL; ++j)
#pragma unroll
    for (int b = 0; b < S; ++b) t[j * S + b] = v[j][b];
  st_span<float, CPL * S>(base + ((size_t)r.a * io.C + r.u0) * S, t);
}

// lane's weights w[e][u0 .. u0+CPL)[0..LM) of one per-edge weight array, as raw 32-bit words
template <typename T, int CPL, int LM>
struct WSpan {
  static constexpr int N = CPL * LM;
  static constexpr int NB = N * (int)sizeof(T);
  static constexpr int NW = NB / 4;
};

template <typename T, int CPL, int LM>
__device__ __forceinline__ void ld_w_raw(const T* arr, int ld, int col0, int e, const RowCtx& r,
                                         uint32_t (&w)[WSpan<T, CPL, LM>::NW]) {
  if (r.act) ld_words<WSpan<T, CPL, LM>::NB>(arr + (size_t)e * ld + col0 + r.u0 * LM, w);
  else {
#pragma unroll
    for (int q = 0; q < WSpan<T, CPL, LM>::NW; ++q) w[q] = 0u;
  }
}

template <typename T, int CPL, int LM>
__device__ __forceinline__ void st_w(T* arr, int ld, int col0, int e, const RowCtx& r, const float (&w)[CPL * LM]) {
  if (r.act) st_span<T, CPL * LM>(arr + (size_t)e * ld + col0 + r.u0 * LM, w);
}

// lane's CPL values of a per-edge adjoint row (activation type), kept as raw
// 32-bit words until the arithmetic so that a batch's loads are not
// serialised behind conversions.  The row pitch and column offset are even
// (every activation array is allocated with pitches that are multiples of 8
// elements), so a lane's CPL (even) values are whole aligned words.
template <typename T, int CPL>
struct SbarW {
  static constexpr int NB = CPL * (int)sizeof(T);
  static constexpr int NW = NB / 4;
};
template <typename T, int CPL>
__device__ __forceinline__ void ld_sbar(const void* sbar, int ld, int e, const RowCtx& r,
                                        uint32_t (&w)[SbarW<T, CPL>::NW]) {
  if (r.act) ld_words<SbarW<T, CPL>::NB>(reinterpret_cast<const T*>(sbar) + (size_t)e * ld + r.u0, w);
  else {
#pragma unroll
    for (int q = 0; q < SbarW<T, CPL>::NW; ++q) w[q] = 0u;
  }
}
// the same values as CPL separate element loads (raw bits in the low bits of each word)
template <typename T, int CPL>
__device__ __forceinline__ void ld_sbar_el(const void* sbar, int ld, int e, const RowCtx& r, uint32_t (&w)[CPL]) {
  const T* p = reinterpret_cast<const T*>(sbar) + (size_t)e * ld + r.u0;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    if constexpr (sizeof(T) == 2) w[j] = r.act ? (uint32_t)reinterpret_cast<const unsigned short*>(p)[j] : 0u;
    else w[j] = r.act ? reinterpret_cast<const uint32_t*>(p)[j] : 0u;
  }
}
__device__ __forceinline__ float2 sbar_el_pair(const uint32_t* w, int p, bool half) {
  return half ? make_float2(__uint_as_float(w[2 * p] << 16), __uint_as_float(w[2 * p + 1] << 16))
              : make_float2(__uint_as_float(w[2 * p]), __uint_as_float(w[2 * p + 1]));
}
// channels (2p, 2p + 1) of the lane's raw sbar words
template <typename T, int CPL>
__device__ __forceinline__ float2 sbar_pair(const uint32_t (&w)[SbarW<T, CPL>::NW], int p) {
  if constexpr (sizeof(T) == 2) {
    const uint32_t x = w[p];   // bf16 -> float is exact: the bf16 bits are the upper half of the float
    return make_float2(__uint_as_float(x << 16), __uint_as_float(x & 0xffff0000u));
  } else {
    return make_float2(__uint_as_float(w[2 * p]), __uint_as_float(w[2 * p + 1]));
  }
}

// Edges of a segment in batches of D: the loads of a whole batch are issued
// before any of its arithmetic, so each warp keeps D edges of loads in flight.
template <int D, typename Load, typename Comp>
__device__ __forceinline__ void edge_batches(int cnt, Load&& load, Comp&& comp) {
  for (int k0 = 0; k0 < cnt; k0 += D) {
    const int nb = min(D, cnt - k0);
#pragma unroll
    for (int u = 0; u < D; ++u)
      if (u < nb) load(u, k0 + u);
#pragma unroll
    for (int u = 0; u < D; ++u)
      if (u < nb) comp(u, k0 + u);
  }
}

constexpr int kBatchLight = 8;   // edges per batch in passes with one weight array
constexpr int kBatchHeavy = 4;   // first pass of the layer-1 adjoint (weights + two sbar, most live state)
constexpr int kBatchLast = 6;  // both passes of the last-layer adjoint (measured: 6 beats 8 and 12 there)

// Gamma-type environment sum over the row: G[j][b] = sum_e w[e][j][l(b)] Y[e][b]
template <typename T, int LMAX, int CPL>
__device__ __forceinline__ void env_sum(const RowIO& io, const RowCtx& r, const YStage<(LMAX + 1) * (LMAX + 1)>& ys,
                                        const T* warr, int ldw, int col0, float (&G)[CPL][(LMAX + 1) * (LMAX + 1)],
                                        int& staged) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  using WS = WSpan<T, CPL, LM>;
  float2 G2[CPL / 2][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) G2[p][b] = bc(0.0f);
  for (int sb = r.rb; sb < r.re; sb += kYSeg) {
    const int cnt = min(kYSeg, r.re - sb);
    ys.load(io.Y, sb, cnt, r.lane);
    staged = sb;
    uint32_t raw[kBatchLight][WS::NW];
    edge_batches<kBatchLight>(
        cnt, [&](int u, int k) { ld_w_raw<T, CPL, LM>(warr, ldw, col0, sb + k, r, raw[u]); },
        [&](int u, int k) {
          float y[S], w[WS::N];
          ys.get(k, y);
          unpack_span<T, WS::N>(raw[u], w);
#pragma unroll
          for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
            for (int b = 0; b < S; ++b) {
              const int l = lof<LMAX>(b);
              G2[p][b] = fma2(pk(w[2 * p * LM + l], w[(2 * p + 1) * LM + l]), bc(y[b]), G2[p][b]);
            }
        });
  }
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) {
      G[2 * p][b] = G2[p][b].x;
      G[2 * p + 1][b] = G2[p][b].y;
    }
}

// s[e][u] = sum_p w0[e][u][l(p)] Y[e][p] M[u][p]  (scalar output of a product), written at column xs_off + u
template <typename T, int LMAX, int CPL>
__device__ __forceinline__ void scalar_out(const RowIO& io, const RowCtx& r, const YStage<(LMAX + 1) * (LMAX + 1)>& ys,
                                           const float (&M)[CPL][(LMAX + 1) * (LMAX + 1)], int staged) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  using WS = WSpan<T, CPL, LM>;
  const T* W01 = reinterpret_cast<const T*>(io.W01);
  T* xs = reinterpret_cast<T*>(io.xs);
  const int nseg = (r.re - r.rb + kYSeg - 1) / kYSeg;
  for (int q = nseg - 1; q >= 0; --q) {   // last segment first: it is still staged
    const int sb = r.rb + q * kYSeg, cnt = min(kYSeg, r.re - sb);
    if (sb != staged) ys.load(io.Y, sb, cnt, r.lane);
    staged = sb;
    uint32_t raw[kBatchLight][WS::NW];
    edge_batches<kBatchLight>(
        cnt, [&](int u, int k) { ld_w_raw<T, CPL, LM>(W01, io.ld01, 0, sb + k, r, raw[u]); },
        [&](int u, int k) {
          const int e = sb + k;
          float y[S], w[WS::N];
          ys.get(k, y);
          unpack_span<T, WS::N>(raw[u], w);
#pragma unroll
          for (int jp = 0; jp < CPL / 2; ++jp) {
            float2 t[LM];
#pragma unroll
            for (int l = 0; l < LM; ++l) t[l] = bc(0.0f);
#pragma unroll
            for (int p = 0; p < S; ++p) t[lof<LMAX>(p)] = fma2(bc(y[p]), pk(M[2 * jp][p], M[2 * jp + 1][p]), t[lof<LMAX>(p)]);
            float2 sv = bc(0.0f);
#pragma unroll
            for (int l = 0; l < LM; ++l) sv = fma2(pk(w[2 * jp * LM + l], w[(2 * jp + 1) * LM + l]), t[l], sv);
            if (r.act) {
              T* o = xs + (size_t)e * io.ldxs + io.xs_off + r.u0 + 2 * jp;
              o[0] = to_act2<T>(sv.x);
              o[1] = to_act2<T>(sv.y);
            }
          }
        });
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// forward, layer 1 of a two-layer model: Gamma^1 and s^1 = V^1_{0e}
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int CPL>
__global__ void __launch_bounds__(32 * kRowWarps) row_fwd_mid_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  __shared__ __align__(16) float ysm[kRowWarps * kYSeg * YStage<S>::P];
  RowCtx r;
  if (!row_ctx<CPL>(io, r)) return;
  const YStage<S> ys{ysm + (threadIdx.x >> 5) * kYSeg * YStage<S>::P};
  const int nw = io.C * (LMAX + 1);
  int staged = -1;
  float G[CPL][S];
  env_sum<T, LMAX, CPL>(io, r, ys, reinterpret_cast<const T*>(io.W01), io.ld01, nw, G, staged);
#pragma unroll
  for (int j = 0; j < CPL; ++j)
#pragma unroll
    for (int b = 0; b < S; ++b) G[j][b] *= tp.nu;
  st_atom<CPL, S>(io.G1, io, r, G);
  // only the scalar output c = 0 is needed here: M0[p] = sum_b W[p][b][0] G_b
  float M0[CPL][S];
#pragma unroll
  for (int j = 0; j < CPL; ++j)
#pragma unroll
    for (int p = 0; p < S; ++p) {
      float s = 0.0f;
#pragma unroll
      for (int b = 0; b < S; ++b)
        if (tp_nonzero(p, b, 0)) s += tp.W1[(p * S + b) * S + 0] * G[j][b];
      M0[j][p] = s;
    }
  scalar_out<T, LMAX, CPL>(io, r, ys, M0, staged);
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
      if (!tp_any_c(p, b, S)) continue;
      float q = 0.0f;
#pragma unroll
      for (int c = 0; c < S; ++c)
        if (tp_nonzero(p, b, c)) q += tp.W1[(p * S + b) * S + c] * cg[c];
      t += G1[b] * q;
    }
    T2[p] = t;
  }
}

// ---------------------------------------------------------------------------
// forward, last layer NL: Gamma^NL and s^NL
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int NL, int CPL>
__global__ void __launch_bounds__(32 * kRowWarps) row_fwd_last_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  __shared__ __align__(16) float ysm[kRowWarps * kYSeg * YStage<S>::P];
  RowCtx r;
  if (!row_ctx<CPL>(io, r)) return;
  const YStage<S> ys{ysm + (threadIdx.x >> 5) * kYSeg * YStage<S>::P};
  const int nw = io.C * (LMAX + 1);
  const T* wsrc = (NL == 1) ? reinterpret_cast<const T*>(io.W01) : reinterpret_cast<const T*>(io.w2);
  const int ldw = (NL == 1) ? io.ld01 : io.ld2;
  const int col0 = (NL == 1) ? nw : 0;
  int staged = -1;
  float G[CPL][S];
  env_sum<T, LMAX, CPL>(io, r, ys, wsrc, ldw, col0, G, staged);
  float Tv[CPL][S];
  float G1[CPL][S];
  if constexpr (NL == 2) ld_atom<CPL, S>(io.G1, io, r, G1);
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    float cg[S];
#pragma unroll
    for (int b = 0; b < S; ++b) {
      G[j][b] *= tp.nu;
      cg[b] = tp.clast[b] * G[j][b];
    }
    if constexpr (NL == 2) {
      make_T2<S>(tp, G1[j], cg, Tv[j]);
    } else {
#pragma unroll
      for (int b = 0; b < S; ++b) Tv[j][b] = cg[b];
    }
  }
  st_atom<CPL, S>((NL == 1) ? io.G1 : io.G2, io, r, G);
  scalar_out<T, LMAX, CPL>(io, r, ys, Tv, staged);
}

// ---------------------------------------------------------------------------
// adjoint, last layer NL.  Given sbar^NL[e][u]:
//   NL = 2:  Gamma^2bar = clast . (M^1^T Q2);  wbar^2 and Ybar (=) from Gamma^2bar
//   NL = 1:  Gamma^1bar_b = clast_b sum_e sbar_e V^0_{e,b};  V^0bar = sbar clast Gamma^1;
//            wbar^0 and its Ybar part (=) in the first pass, wbar^1 and its Ybar part (+=) in the second
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int NL, int CPL>
__global__ void __launch_bounds__(32 * kRowWarps) row_bwd_last_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  __shared__ __align__(16) float ysm[kRowWarps * kYSeg * YStage<S>::P];
  RowCtx r;
  if (!row_ctx<CPL>(io, r)) return;
  const YStage<S> ys{ysm + (threadIdx.x >> 5) * kYSeg * YStage<S>::P};
  const int nw = io.C * LM;
  const T* W01 = reinterpret_cast<const T*>(io.W01);
  const void* sbar = (NL == 1) ? io.sbar1 : io.sbar2;
  const int lds = (NL == 1) ? io.ld_sbar1 : io.ld_sbar2;
  T* wb01 = reinterpret_cast<T*>(io.wbar01);
  // NL = 1: V^0bar_{e,a} = sbar_e cG_a with cG = clast Gamma^1 (known before the pass)
  float cG[CPL][S];
  if constexpr (NL == 1) {
    ld_atom<CPL, S>(io.G1, io, r, cG);
#pragma unroll
    for (int j = 0; j < CPL; ++j)
#pragma unroll
      for (int b = 0; b < S; ++b) cG[j][b] *= tp.clast[b];
  }
  // pass 1: Q[a] = sum_e sbar_e V^0_{e,a}  (+ NL = 1: wbar^0, Ybar from w^0)
  float2 Q2[CPL / 2][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) Q2[p][b] = bc(0.0f);
  int staged = -1;
  using WS = WSpan<T, CPL, LM>;
  for (int sb = r.rb; sb < r.re; sb += kYSeg) {
    const int cnt = min(kYSeg, r.re - sb);
    ys.load(io.Y, sb, cnt, r.lane);
    staged = sb;
    uint32_t raw[kBatchLast][WS::NW];
    uint32_t sraw[kBatchLast][CPL];
    edge_batches<kBatchLast>(
        cnt,
        [&](int u, int k) {
          ld_w_raw<T, CPL, LM>(W01, io.ld01, 0, sb + k, r, raw[u]);
          ld_sbar_el<T, CPL>(sbar, lds, sb + k, r, sraw[u]);
        },
        [&](int u, int k) {
          const int e = sb + k;
          float y[S], w0[WS::N], g0[WS::N];
          float2 yc2[S];
          ys.get(k, y);
          unpack_span<T, WS::N>(raw[u], w0);
#pragma unroll
          for (int b = 0; b < S; ++b) yc2[b] = bc(0.0f);
#pragma unroll
          for (int p = 0; p < CPL / 2; ++p) {
            const float2 sj = sbar_el_pair(sraw[u], p, sizeof(T) == 2);
            float2 t[LM], g[LM];
#pragma unroll
            for (int l = 0; l < LM; ++l) {
              t[l] = mul2(sj, pk(w0[2 * p * LM + l], w0[(2 * p + 1) * LM + l]));
              g[l] = bc(0.0f);
            }
#pragma unroll
            for (int b = 0; b < S; ++b) Q2[p][b] = fma2(t[lof<LMAX>(b)], bc(y[b]), Q2[p][b]);
            if constexpr (NL == 1) {
#pragma unroll
              for (int b = 0; b < S; ++b) {
                const int l = lof<LMAX>(b);
                const float2 v0b = mul2(sj, pk(cG[2 * p][b], cG[2 * p + 1][b]));
                g[l] = fma2(v0b, bc(y[b]), g[l]);
                yc2[b] = fma2(pk(w0[2 * p * LM + l], w0[(2 * p + 1) * LM + l]), v0b, yc2[b]);
              }
#pragma unroll
              for (int l = 0; l < LM; ++l) {
                g0[2 * p * LM + l] = g[l].x;
                g0[(2 * p + 1) * LM + l] = g[l].y;
              }
            }
          }
          if constexpr (NL == 1) {
            float yc[S];
#pragma unroll
            for (int b = 0; b < S; ++b) yc[b] = yc2[b].x + yc2[b].y;
            st_w<T, CPL, LM>(wb01, io.ld_wbar01, 0, e, r, g0);
            warp_channel_sum<S>(yc, r.lane, io.Ybar[0] + (size_t)e * S);
          }
        });
  }
  float Q[CPL][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) {
      Q[2 * p][b] = Q2[p][b].x;
      Q[2 * p + 1][b] = Q2[p][b].y;
    }
  // Gamma^NL bar, pre-scaled by nu
  float Gb[CPL][S];
  float G1[CPL][S];
  if constexpr (NL == 2) ld_atom<CPL, S>(io.G1, io, r, G1);
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    if constexpr (NL == 2) {
#pragma unroll
      for (int b = 0; b < S; ++b) Gb[j][b] = 0.0f;
#pragma unroll
      for (int p = 0; p < S; ++p)
#pragma unroll
        for (int bp = 0; bp < S; ++bp) {
          if (!tp_any_c(p, bp, S)) continue;
          const float gq = G1[j][bp] * Q[j][p];
#pragma unroll
          for (int b = 0; b < S; ++b)
            if (tp_nonzero(p, bp, b)) Gb[j][b] += tp.W1[(p * S + bp) * S + b] * gq;
        }
#pragma unroll
      for (int b = 0; b < S; ++b) Gb[j][b] *= tp.clast[b] * tp.nu;
    } else {
#pragma unroll
      for (int b = 0; b < S; ++b) Gb[j][b] = tp.clast[b] * Q[j][b] * tp.nu;
    }
  }
  // pass 2: wbar^NL_l = nu sum_{b in l} Gamma^NL bar_b Y_b;  Ybar += sum_u nu w^NL Gamma^NL bar
  T* wbL = (NL == 1) ? wb01 : reinterpret_cast<T*>(io.wbar2);
  const int ldwb = (NL == 1) ? io.ld_wbar01 : io.ld_wbar2;
  const T* wsrc = (NL == 1) ? W01 : reinterpret_cast<const T*>(io.w2);
  const int ldw = (NL == 1) ? io.ld01 : io.ld2;
  const int col0 = (NL == 1) ? nw : 0;
  const int nseg = (r.re - r.rb + kYSeg - 1) / kYSeg;
  float* ybar_out = io.Ybar[NL == 1 ? 1 : 0];
  float2 Gb2[CPL / 2][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) Gb2[p][b] = pk(Gb[2 * p][b], Gb[2 * p + 1][b]);
  for (int q = nseg - 1; q >= 0; --q) {
    const int sb = r.rb + q * kYSeg, cnt = min(kYSeg, r.re - sb);
    if (sb != staged) ys.load(io.Y, sb, cnt, r.lane);
    staged = sb;
    uint32_t raw[kBatchLast][WS::NW];
    edge_batches<kBatchLast>(
        cnt, [&](int u, int k) { ld_w_raw<T, CPL, LM>(wsrc, ldw, col0, sb + k, r, raw[u]); },
        [&](int u, int k) {
          const int e = sb + k;
          float y[S], w[WS::N], g[WS::N], yc[S];
          float2 yc2[S];
          ys.get(k, y);
          unpack_span<T, WS::N>(raw[u], w);
#pragma unroll
          for (int b = 0; b < S; ++b) yc2[b] = bc(0.0f);
#pragma unroll
          for (int p = 0; p < CPL / 2; ++p) {
            float2 g2[LM];
#pragma unroll
            for (int l = 0; l < LM; ++l) g2[l] = bc(0.0f);
#pragma unroll
            for (int b = 0; b < S; ++b) {
              const int l = lof<LMAX>(b);
              g2[l] = fma2(Gb2[p][b], bc(y[b]), g2[l]);
              yc2[b] = fma2(pk(w[2 * p * LM + l], w[(2 * p + 1) * LM + l]), Gb2[p][b], yc2[b]);
            }
#pragma unroll
            for (int l = 0; l < LM; ++l) {
              g[2 * p * LM + l] = g2[l].x;
              g[(2 * p + 1) * LM + l] = g2[l].y;
            }
          }
#pragma unroll
          for (int b = 0; b < S; ++b) yc[b] = yc2[b].x + yc2[b].y;
          st_w<T, CPL, LM>(wbL, ldwb, col0, e, r, g);
          warp_channel_sum<S>(yc, r.lane, ybar_out + (size_t)e * S);
        });
  }
}

// ---------------------------------------------------------------------------
// adjoint, layer 1 of a two-layer model (factorised, see above):
//   pass 1: Q1 = sum_e sbar^1 V^0, Q2 = sum_e sbar^2 V^0
//   per atom: T1, T2 (from Gamma^1, Gamma^2) and Gamma^1bar (pre-scaled by nu)
//   pass 2: V^0bar = sbar^2 T2 + sbar^1 T1;  wbar^0_l = sum_m V^0bar Y;
//           wbar^1_l = nu sum_m Gamma^1bar Y;  Ybar = sum_u (w^0 V^0bar + nu w^1 Gamma^1bar)
// The second pass reads the row's w^0 and sbar again (from L2: the row was
// just read) so that each pass keeps only half the per-channel state.
// ---------------------------------------------------------------------------
template <typename T, int LMAX, int CPL>
// (at most 128 registers: four blocks per SM; measured faster than the unbounded 157)
__global__ void __launch_bounds__(32 * kRowWarps, 4) row_bwd_mid_kernel(RowIO io, TPConst tp) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  constexpr int LM = LMAX + 1;
  __shared__ __align__(16) float ysm[kRowWarps * kYSeg * YStage<S>::P];
  RowCtx r;
  if (!row_ctx<CPL>(io, r)) return;
  const YStage<S> ys{ysm + (threadIdx.x >> 5) * kYSeg * YStage<S>::P};
  const int nw = io.C * LM;
  const T* W01 = reinterpret_cast<const T*>(io.W01);
  T* wb = reinterpret_cast<T*>(io.wbar01);
  using WS = WSpan<T, CPL, LM>;
  float2 Q1p[CPL / 2][S], Q2p[CPL / 2][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) { Q1p[p][b] = bc(0.0f); Q2p[p][b] = bc(0.0f); }
  int staged = -1;
  for (int sb = r.rb; sb < r.re; sb += kYSeg) {
    const int cnt = min(kYSeg, r.re - sb);
    ys.load(io.Y, sb, cnt, r.lane);
    staged = sb;
    uint32_t raw[kBatchLight][WS::NW];
    uint32_t s1r[kBatchLight][SbarW<T, CPL>::NW], s2r[kBatchLight][SbarW<T, CPL>::NW];
    edge_batches<kBatchLight>(
        cnt,
        [&](int u, int k) {
          ld_w_raw<T, CPL, LM>(W01, io.ld01, 0, sb + k, r, raw[u]);
          ld_sbar<T, CPL>(io.sbar1, io.ld_sbar1, sb + k, r, s1r[u]);
          ld_sbar<T, CPL>(io.sbar2, io.ld_sbar2, sb + k, r, s2r[u]);
        },
        [&](int u, int k) {
          float y[S], w0[WS::N];
          ys.get(k, y);
          unpack_span<T, WS::N>(raw[u], w0);
#pragma unroll
          for (int p = 0; p < CPL / 2; ++p) {
            const float2 s1 = sbar_pair<T, CPL>(s1r[u], p);
            const float2 s2 = sbar_pair<T, CPL>(s2r[u], p);
#pragma unroll
            for (int b = 0; b < S; ++b) {
              const int l = lof<LMAX>(b);
              const float2 v0 = mul2(pk(w0[2 * p * LM + l], w0[(2 * p + 1) * LM + l]), bc(y[b]));
              Q1p[p][b] = fma2(s1, v0, Q1p[p][b]);
              Q2p[p][b] = fma2(s2, v0, Q2p[p][b]);
            }
          }
        });
  }
  float Q1[CPL][S], Q2[CPL][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) {
      Q1[2 * p][b] = Q1p[p][b].x; Q1[2 * p + 1][b] = Q1p[p][b].y;
      Q2[2 * p][b] = Q2p[p][b].x; Q2[2 * p + 1][b] = Q2p[p][b].y;
    }
  // per atom: T1, T2, Gamma^1bar
  float T1[CPL][S], T2[CPL][S], G1b[CPL][S];
  {
    float G1[CPL][S], cg2[CPL][S];
    ld_atom<CPL, S>(io.G1, io, r, G1);
    ld_atom<CPL, S>(io.G2, io, r, cg2);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
#pragma unroll
      for (int b = 0; b < S; ++b) cg2[j][b] *= tp.clast[b];
      make_T2<S>(tp, G1[j], cg2[j], T2[j]);
#pragma unroll
      for (int p = 0; p < S; ++p) {
        float t = 0.0f;
#pragma unroll
        for (int b = 0; b < S; ++b)
          if (tp_nonzero(p, b, 0)) t += tp.W1[(p * S + b) * S + 0] * G1[j][b];
        T1[j][p] = t;
      }
      // gather order (one output at a time) keeps few values live
#pragma unroll
      for (int b = 0; b < S; ++b) {
        float acc = 0.0f;
#pragma unroll
        for (int p = 0; p < S; ++p) {
          if (tp_any_c(p, b, S)) {
            float q = 0.0f;
#pragma unroll
            for (int c = 0; c < S; ++c)
              if (tp_nonzero(p, b, c)) q += tp.W1[(p * S + b) * S + c] * cg2[j][c];
            acc += Q2[j][p] * q;
          }
          if (tp_nonzero(p, b, 0)) acc += Q1[j][p] * tp.W1[(p * S + b) * S + 0];
        }
        G1b[j][b] = acc * tp.nu;
      }
    }
  }
  float2 T1p[CPL / 2][S], T2p[CPL / 2][S], G1bp[CPL / 2][S];
#pragma unroll
  for (int p = 0; p < CPL / 2; ++p)
#pragma unroll
    for (int b = 0; b < S; ++b) {
      T1p[p][b] = pk(T1[2 * p][b], T1[2 * p + 1][b]);
      T2p[p][b] = pk(T2[2 * p][b], T2[2 * p + 1][b]);
      G1bp[p][b] = pk(G1b[2 * p][b], G1b[2 * p + 1][b]);
    }
  const int nseg = (r.re - r.rb + kYSeg - 1) / kYSeg;
  for (int q = nseg - 1; q >= 0; --q) {
    const int sb = r.rb + q * kYSeg, cnt = min(kYSeg, r.re - sb);
    if (sb != staged) ys.load(io.Y, sb, cnt, r.lane);
    staged = sb;
    uint32_t raw0[kBatchHeavy][WS::NW], raw1[kBatchHeavy][WS::NW];
    uint32_t s1r[kBatchHeavy][SbarW<T, CPL>::NW], s2r[kBatchHeavy][SbarW<T, CPL>::NW];
    edge_batches<kBatchHeavy>(
        cnt,
        [&](int u, int k) {
          ld_w_raw<T, CPL, LM>(W01, io.ld01, 0, sb + k, r, raw0[u]);
          ld_w_raw<T, CPL, LM>(W01, io.ld01, nw, sb + k, r, raw1[u]);
          ld_sbar<T, CPL>(io.sbar1, io.ld_sbar1, sb + k, r, s1r[u]);
          ld_sbar<T, CPL>(io.sbar2, io.ld_sbar2, sb + k, r, s2r[u]);
        },
        [&](int u, int k) {
          const int e = sb + k;
          float y[S], w0[WS::N], w1[WS::N], g0[WS::N], g1[WS::N], yc[S];
          float2 yc2[S];
          ys.get(k, y);
          unpack_span<T, WS::N>(raw0[u], w0);
          unpack_span<T, WS::N>(raw1[u], w1);
#pragma unroll
          for (int b = 0; b < S; ++b) yc2[b] = bc(0.0f);
#pragma unroll
          for (int p = 0; p < CPL / 2; ++p) {
            const float2 s1 = sbar_pair<T, CPL>(s1r[u], p);
            const float2 s2 = sbar_pair<T, CPL>(s2r[u], p);
            float2 a0[LM], a1[LM];
#pragma unroll
            for (int l = 0; l < LM; ++l) { a0[l] = bc(0.0f); a1[l] = bc(0.0f); }
#pragma unroll
            for (int b = 0; b < S; ++b) {
              const int l = lof<LMAX>(b);
              const float2 yy = bc(y[b]);
              const float2 v0b = fma2(s2, T2p[p][b], mul2(s1, T1p[p][b]));
              a0[l] = fma2(v0b, yy, a0[l]);
              a1[l] = fma2(G1bp[p][b], yy, a1[l]);
              yc2[b] = fma2(pk(w0[2 * p * LM + l], w0[(2 * p + 1) * LM + l]), v0b, yc2[b]);
              yc2[b] = fma2(pk(w1[2 * p * LM + l], w1[(2 * p + 1) * LM + l]), G1bp[p][b], yc2[b]);
            }
#pragma unroll
            for (int l = 0; l < LM; ++l) {
              g0[2 * p * LM + l] = a0[l].x; g0[(2 * p + 1) * LM + l] = a0[l].y;
              g1[2 * p * LM + l] = a1[l].x; g1[(2 * p + 1) * LM + l] = a1[l].y;
            }
          }
#pragma unroll
          for (int b = 0; b < S; ++b) yc[b] = yc2[b].x + yc2[b].y;
          st_w<T, CPL, LM>(wb, io.ld_wbar01, 0, e, r, g0);
          st_w<T, CPL, LM>(wb, io.ld_wbar01, nw, e, r, g1);
          warp_channel_sum<S>(yc, r.lane, io.Ybar[1] + (size_t)e * S);
        });
  }
}

// ---------------------------------------------------------------------------
namespace {
template <typename T, int CPL>
void row_fwd_cpl(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st) {
  dim3 grid((io.na + kRowWarps - 1) / kRowWarps), block(32 * kRowWarps);
  if (layer < nl) {
    if (lmax == 1) row_fwd_mid_kernel<T, 1, CPL><<<grid, block, 0, st>>>(io, tp);
    else row_fwd_mid_kernel<T, 2, CPL><<<grid, block, 0, st>>>(io, tp);
  } else if (nl == 1) {
    if (lmax == 1) row_fwd_last_kernel<T, 1, 1, CPL><<<grid, block, 0, st>>>(io, tp);
    else row_fwd_last_kernel<T, 2, 1, CPL><<<grid, block, 0, st>>>(io, tp);
  } else {
    if (lmax == 1) row_fwd_last_kernel<T, 1, 2, CPL><<<grid, block, 0, st>>>(io, tp);
    else row_fwd_last_kernel<T, 2, 2, CPL><<<grid, block, 0, st>>>(io, tp);
  }
}

template <typename T, int CPL>
void row_bwd_cpl(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st) {
  dim3 grid((io.na + kRowWarps - 1) / kRowWarps), block(32 * kRowWarps);
  if (layer < nl) {
    if (lmax == 1) row_bwd_mid_kernel<T, 1, CPL><<<grid, block, 0, st>>>(io, tp);
    else row_bwd_mid_kernel<T, 2, CPL><<<grid, block, 0, st>>>(io, tp);
  } else if (nl == 1) {
    if (lmax == 1) row_bwd_last_kernel<T, 1, 1, CPL><<<grid, block, 0, st>>>(io, tp);
    else row_bwd_last_kernel<T, 2, 1, CPL><<<grid, block, 0, st>>>(io, tp);
  } else {
    if (lmax == 1) row_bwd_last_kernel<T, 1, 2, CPL><<<grid, block, 0, st>>>(io, tp);
    else row_bwd_last_kernel<T, 2, 2, CPL><<<grid, block, 0, st>>>(io, tp);
  }
}
}  // namespace

// Channels per lane: 2 up to 64 channels (lanes >= C/2 idle below 64), 4 for 128.
template <typename T>
void row_fwd(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st) {
  if (io.na <= 0) return;
  if (io.C > 64) row_fwd_cpl<T, 4>(layer, nl, lmax, io, tp, st);
  else row_fwd_cpl<T, 2>(layer, nl, lmax, io, tp, st);
}

template <typename T>
void row_bwd(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st) {
  if (io.na <= 0) return;
  if (io.C > 64) row_bwd_cpl<T, 4>(layer, nl, lmax, io, tp, st);
  else row_bwd_cpl<T, 2>(layer, nl, lmax, io, tp, st);
}

template void row_fwd<float>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_fwd<bf16>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_bwd<float>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);
template void row_bwd<bf16>(int, int, int, const RowIO&, const TPConst&, cudaStream_t);

}  // namespace alg
