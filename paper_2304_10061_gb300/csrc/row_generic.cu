// Environment sums and tensor products for any number of layers (Eq. 1), the
// path for models the specialised row kernels do not take (three layers,
// whose middle layers carry features of either parity; l_max 3).
//
// With V^0_e = w^0_e (x) Y_e and V^L_e = V^{L-1}_e (x) Gamma^{i,L} channel by
// channel, every product is linear in V^0_e, so for centre i and channel u
//   V^L_e = V^0_e M^1 M^2 ... M^L,   M^k[a][c] = sum_b W^k[a][b][c] Gamma^k[b],
// and the scalar output of layer L is
//   s^L_e = V^L_e[0e] = sum_a w^0_{e,l(a)} Y_e[a] Q^L[a],
//   Q^L = M^1 (M^2 (... (M^L e_0))),
// a per-atom vector over the S harmonic components (e_0 picks the 0e output;
// the last layer's tensor has that output only).  So per edge the work is
// O(S) per channel, and per atom it is one matrix-vector chain over the
// nonzeros of the layer tensors.  The adjoint, given sbar^L_e:
//   Qbar^L[a]     = sum_e sbar^L_e w^0_{e,l(a)} Y_e[a]                       (per atom)
//   Gammabar^k[b] += sum_{a,c} W^k[a][b][c] rbar_k[a] r_{k+1}[c],   k <= L  (back along the chain,
//   rbar_{k+1}[c] = sum_{a,b} W^k[a][b][c] rbar_k[a] Gamma^k[b],            rbar_1 = Qbar^L,
//                                                                             r_k = M^k ... M^L e_0)
//   wbar^L_{e,l}  = nu sum_{m} Gammabar^L[lm] Y_e[lm]        (once Gammabar^L is complete)
//   w^0bar_{e,l}  = sum_L sum_{a in l} sbar^L_e Y_e[a] Q^L[a]
//   Ybar_e[a]     = sum_L sum_u (sbar^L_e w^0_{e,l(a)} Q^L[a] + nu w^L_{e,l(a)} Gammabar^L[a])
// Layers are processed for L = nl, nl-1, ..., 1 (the order in which the sbar^L
// arrive): Gammabar^L is complete once every layer >= L has been processed, so
// wbar^L is written then; w^0bar and Ybar, sums over all layers, are formed
// once, after layer 1.
//
// Layout: per atom [atom][channel][S] float32; per edge the activation-type
// arrays of the MLP side (w, s, sbar, wbar) and float32 Y / Ybar / w^0bar.
// Row kernels: one warp per centre atom with C / 32 channels per lane (the
// environment sums, s, Qbar, the upper layers' wbar: a lane's harmonics loads
// serve all its channels), or, for the per-edge adjoint that combines every
// layer, one block per centre atom and one thread per channel; per-atom sums
// are register accumulations over the row (deterministic), the channel sums of
// Ybar are warp halving sums and a fixed-order sum over the warps; l_max is a
// template parameter, so every per-edge vector lives in registers.  Chain kernels: one
// thread per (atom, channel), unrolled at compile time over the candidate
// nonzeros of the layer tensors.  Which entries of a fused tensor can be
// nonzero is fixed by l_max and the layer irreps: the paths allowed by the
// triangle and parity rules, and within a path's real coupling block the
// entries with |m3| = |m1| + |m2| or ||m1| - |m2||, whose sine/cosine types
// multiply to the block's type ((-1)^(l1+l2+l3): real harmonics with m < 0 are
// the sine type).  So every vector index is a compile-time constant (the
// vectors live in registers) and the tensor values are launch parameters
// (constant-bank operands of the multiply-adds); the host checks that every
// nonzero of the model's tensors is a candidate.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "amax.cuh"
#include "internal.h"

namespace alg {

namespace {

template <typename T> __device__ __forceinline__ float gld(const T* p);
template <> __device__ __forceinline__ float gld<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float gld<bf16>(const bf16* p) { return __bfloat162float(*p); }
template <typename T> __device__ __forceinline__ void gst(T* p, float v);
template <> __device__ __forceinline__ void gst<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void gst<bf16>(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

__host__ __device__ constexpr int l_of(int a) { return a < 1 ? 0 : (a < 4 ? 1 : (a < 9 ? 2 : 3)); }

// the LM = l_max + 1 weights of one channel: one vector access when LM == 4 (the
// rows are padded to 8 elements and the columns start at multiples of LM, so
// channel u's group starts at a multiple of 4 elements)
template <typename T, int LM>
__device__ __forceinline__ void load_lm(const T* p, float (&x)[LM]) {
  if constexpr (LM == 4 && sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if constexpr (LM == 4 && sizeof(T) == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
    x[0] = lo.x; x[1] = lo.y; x[2] = hi.x; x[3] = hi.y;
  } else {
#pragma unroll
    for (int l = 0; l < LM; ++l) x[l] = gld(p + l);
  }
}
template <typename T, int LM>
__device__ __forceinline__ void store_lm(T* p, const float (&x)[LM]) {
  if constexpr (LM == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else if constexpr (LM == 4 && sizeof(T) == 2) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(x[0], x[1]), hi = __floats2bfloat162_rn(x[2], x[3]);
    uint2 v;
    v.x = *reinterpret_cast<const unsigned*>(&lo);
    v.y = *reinterpret_cast<const unsigned*>(&hi);
    *reinterpret_cast<uint2*>(p) = v;
  } else {
#pragma unroll
    for (int l = 0; l < LM; ++l) gst(p + l, x[l]);
  }
}

// an edge's S harmonics (rows of S floats, 16-byte aligned when S is a multiple of 4)
template <int S>
__device__ __forceinline__ void load_y(const float* p, float (&y)[S]) {
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int k = 0; k < S / 4; ++k) {
      const float4 v = *reinterpret_cast<const float4*>(p + 4 * k);
      y[4 * k] = v.x; y[4 * k + 1] = v.y; y[4 * k + 2] = v.z; y[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) y[a] = p[a];
  }
}

// Warp sums of 16 values by recursive halving: at each of the five steps a lane
// sends the half of its remaining values that its partner keeps.  Returns, in
// every lane, the warp sum of component lane / 2 (16 shuffles instead of 80).
__device__ __forceinline__ float warp_sum16(float (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;   // this lane keeps the upper half
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

constexpr int kChainThreads = 128;   // (atom, channel) pairs per block of the chain kernels

// ---- the layer irreps and candidate nonzeros at compile time ----
struct IrSet {               // irreps (l, parity), sorted by l, even before odd
  int n = 0;
  int l[8] = {};
  int p[8] = {};
};

__host__ __device__ constexpr int iabs(int x) { return x < 0 ? -x : x; }
__host__ __device__ constexpr int imin(int a, int b) { return a < b ? a : b; }

__host__ __device__ constexpr IrSet ir_natural(int lmax) {
  IrSet s{};
  for (int l = 0; l <= lmax; ++l) {
    s.l[s.n] = l;
    s.p[s.n] = (l & 1) ? -1 : 1;
    ++s.n;
  }
  return s;
}

// the irreps of the products of `in` with the harmonics up to l_max, truncated at l_max
__host__ __device__ constexpr IrSet ir_products(const IrSet& in, int lmax) {
  bool has[kMaxLmax + 1][2] = {};
  for (int k = 0; k < in.n; ++k)
    for (int l2 = 0; l2 <= lmax; ++l2)
      for (int lo = iabs(in.l[k] - l2); lo <= imin(in.l[k] + l2, lmax); ++lo)
        has[lo][in.p[k] * ((l2 & 1) ? -1 : 1) == 1 ? 0 : 1] = true;
  IrSet s{};
  for (int l = 0; l <= lmax; ++l)
    for (int q = 0; q < 2; ++q)
      if (has[l][q]) {
        s.l[s.n] = l;
        s.p[s.n] = q ? -1 : 1;
        ++s.n;
      }
  return s;
}

// can (l, p) reach the scalar 0e in `steps` more products?
__host__ __device__ constexpr bool ir_reaches_scalar(int l, int p, int steps, int lmax) {
  if (steps == 0) return l == 0 && p == 1;
  IrSet one{};
  one.n = 1;
  one.l[0] = l;
  one.p[0] = p;
  const IrSet o = ir_products(one, lmax);
  for (int k = 0; k < o.n; ++k)
    if (ir_reaches_scalar(o.l[k], o.p[k], steps - 1, lmax)) return true;
  return false;
}

// the features of layer L of an nl-layer model: the products that can still reach 0e
__host__ __device__ constexpr IrSet ir_layer(int lmax, int nl, int L) {
  IrSet s = ir_natural(lmax);
  for (int k = 1; k <= L; ++k) {
    const IrSet o = ir_products(s, lmax);
    IrSet keep{};
    for (int q = 0; q < o.n; ++q)
      if (ir_reaches_scalar(o.l[q], o.p[q], nl - k, lmax)) {
        keep.l[keep.n] = o.l[q];
        keep.p[keep.n] = o.p[q];
        ++keep.n;
      }
    s = keep;
  }
  return s;
}

__host__ __device__ constexpr int ir_dim(const IrSet& s) {
  int d = 0;
  for (int k = 0; k < s.n; ++k) d += 2 * s.l[k] + 1;
  return d;
}

// can the real coupling block (l1, l2, l3) be nonzero at (m1, m2, m3)?
__host__ __device__ constexpr bool coupling_candidate(int l1, int m1, int l2, int m2, int l3, int m3) {
  const int a = iabs(m1), b = iabs(m2), c = iabs(m3);
  const bool sine = ((m1 < 0) != (m2 < 0)) != (m3 < 0);
  return sine == (((l1 + l2 + l3) & 1) == 1) && (c == a + b || c == iabs(a - b));
}

// Visit the candidate nonzeros (a, b, c) of layer K's tensor in the kernels' order:
// output irrep, input irrep, harmonic degree l2, then m1, m2, m3.
template <typename F>
__host__ __device__ constexpr void for_candidates(int lmax, int nl, int K, F&& f) {
  const IrSet in = ir_layer(lmax, nl, K - 1), out = ir_layer(lmax, nl, K);
  for (int ko = 0, oo = 0; ko < out.n; oo += 2 * out.l[ko] + 1, ++ko)
    for (int ki = 0, oi = 0; ki < in.n; oi += 2 * in.l[ki] + 1, ++ki)
      for (int l2 = 0; l2 <= lmax; ++l2) {
        const int l1 = in.l[ki], lo = out.l[ko];
        if (lo < iabs(l1 - l2) || lo > l1 + l2 || out.p[ko] != in.p[ki] * ((l2 & 1) ? -1 : 1)) continue;
        for (int m1 = -l1; m1 <= l1; ++m1)
          for (int m2 = -l2; m2 <= l2; ++m2)
            for (int m3 = -lo; m3 <= lo; ++m3)
              if (coupling_candidate(l1, m1, l2, m2, lo, m3)) f(oi + l1 + m1, l2 * l2 + l2 + m2, oo + lo + m3);
      }
}

struct CountFn {
  int n = 0;
  __host__ __device__ constexpr void operator()(int, int, int) { ++n; }
};
__host__ __device__ constexpr int n_candidates(int lmax, int nl, int K) {
  CountFn f{};
  for_candidates(lmax, nl, K, f);
  return f.n;
}

template <int N>
struct CandList {
  unsigned char a[N] = {}, b[N] = {}, c[N] = {};
};
template <int N>
struct FillFn {
  CandList<N>* out;
  int q = 0;
  __host__ __device__ constexpr void operator()(int a, int b, int c) {
    out->a[q] = (unsigned char)a;
    out->b[q] = (unsigned char)b;
    out->c[q] = (unsigned char)c;
    ++q;
  }
};
template <int N>
__host__ __device__ constexpr CandList<N> candidates(int lmax, int nl, int K) {
  CandList<N> r{};
  FillFn<N> f{&r};
  for_candidates(lmax, nl, K, f);
  return r;
}

// layer K of an (LMAX, NL) model: its candidates and their offset in the value array
template <int LMAX, int NL, int K>
struct Cand {
  static constexpr int n = n_candidates(LMAX, NL, K);
  static constexpr int off = Cand<LMAX, NL, K - 1>::off + Cand<LMAX, NL, K - 1>::n;
  static constexpr CandList<n> list = candidates<n>(LMAX, NL, K);
  static constexpr int din = ir_dim(ir_layer(LMAX, NL, K - 1)), dout = ir_dim(ir_layer(LMAX, NL, K));
};
template <int LMAX, int NL>
struct Cand<LMAX, NL, 0> {
  static constexpr int n = 0, off = 0;
};
template <class P>
__host__ __device__ constexpr int cand_a(int q) { return P::list.a[q]; }
template <class P>
__host__ __device__ constexpr int cand_b(int q) { return P::list.b[q]; }
template <class P>
__host__ __device__ constexpr int cand_c(int q) { return P::list.c[q]; }

// the values of all layers' candidates, a launch parameter
template <int LMAX, int NL>
struct GenVals {
  static constexpr int n = Cand<LMAX, NL, NL>::off + Cand<LMAX, NL, NL>::n;
  float v[n];
};

template <class F, int... Q>
__device__ __forceinline__ void each_candidate(F&& f, std::integer_sequence<int, Q...>) {
  (f(std::integral_constant<int, Q>{}), ...);
}

// y = M^K x over layer K's candidates, M^K[a][c] = sum_b W^K[a][b][c] G[b]; x = e_0 when E0
template <int LMAX, int NL, int K, bool E0, int D>
__device__ __forceinline__ void chain_mv(const float* v, const float (&G)[D], const float (&x)[kGenMaxD],
                                         float (&y)[kGenMaxD]) {
  using P = Cand<LMAX, NL, K>;
#pragma unroll
  for (int a = 0; a < P::din; ++a) y[a] = 0.0f;
  each_candidate([&](auto q) {
    constexpr int Q = decltype(q)::value;
    constexpr int a = cand_a<P>(Q), b = cand_b<P>(Q), c = cand_c<P>(Q);
    if constexpr (E0) {
      if constexpr (c == 0) y[a] = fmaf(v[P::off + Q], G[b], y[a]);
    } else {
      y[a] = fmaf(v[P::off + Q] * G[b], x[c], y[a]);
    }
  }, std::make_integer_sequence<int, P::n>{});
}

}  // namespace

// Q^L[i][u][:] = M^1 ... M^L e_0
template <int LMAX, int NL, int L>
__global__ void __launch_bounds__(kChainThreads) gen_chain_fwd_kernel(GenRowIO io, const __grid_constant__ GenVals<LMAX, NL> w) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= io.na * io.C) return;
  const size_t o = (size_t)t * S;
  float G[L][S];
#pragma unroll
  for (int k = 0; k < L; ++k)
#pragma unroll
    for (int b = 0; b < S; ++b) G[k][b] = io.G[k + 1][o + b];
  float x[kGenMaxD], y[kGenMaxD];
  chain_mv<LMAX, NL, L, true>(w.v, G[L - 1], x, y);
  if constexpr (L >= 2) {
    chain_mv<LMAX, NL, L - 1, false>(w.v, G[L - 2], y, x);
    if constexpr (L >= 3) {
      chain_mv<LMAX, NL, L - 2, false>(w.v, G[L - 3], x, y);
    }
  }
  const float* q = (L == 2) ? x : y;
  float* out = io.Q[L] + o;
#pragma unroll
  for (int a = 0; a < S; ++a) out[a] = q[a];
}

// Gb[b] += sum over layer K's candidates of W^K[a][b][c] rb[a] r[c] (r = e_0 when E0) and, unless
// !NB, nb[c] = sum W^K[a][b][c] rb[a] G[b]
template <int LMAX, int NL, int K, bool E0, bool NB, int D>
__device__ __forceinline__ void chain_adj(const float* v, const float (&G)[D], const float (&rb)[kGenMaxD],
                                          const float (&r)[kGenMaxD], float (&gb)[D], float (&nb)[kGenMaxD]) {
  using P = Cand<LMAX, NL, K>;
#pragma unroll
  for (int b = 0; b < D; ++b) gb[b] = 0.0f;
  if constexpr (NB) {
#pragma unroll
    for (int c = 0; c < P::dout; ++c) nb[c] = 0.0f;
  }
  each_candidate([&](auto q) {
    constexpr int Q = decltype(q)::value;
    constexpr int a = cand_a<P>(Q), b = cand_b<P>(Q), c = cand_c<P>(Q);
    const float t = v[P::off + Q] * rb[a];
    if constexpr (E0) {
      if constexpr (c == 0) gb[b] += t;
    } else {
      gb[b] = fmaf(t, r[c], gb[b]);
    }
    if constexpr (NB) nb[c] = fmaf(t, G[b], nb[c]);
  }, std::make_integer_sequence<int, P::n>{});
}

// Back along the chain of Q^L: Gammabar^k += ..., k = 1..L
template <int LMAX, int NL, int L>
__global__ void __launch_bounds__(kChainThreads) gen_chain_bwd_kernel(GenRowIO io, const __grid_constant__ GenVals<LMAX, NL> w) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= io.na * io.C) return;
  const size_t o = (size_t)t * S;
  float G[L][S];
#pragma unroll
  for (int k = 0; k < L; ++k)
#pragma unroll
    for (int b = 0; b < S; ++b) G[k][b] = io.G[k + 1][o + b];
  // r_{L+1} = e_0, r_k = M^k r_{k+1}: r[k - 2] holds r_k for k = 2..L
  float r[L > 1 ? L - 1 : 1][kGenMaxD];
  float dummy[kGenMaxD];
  if constexpr (L >= 2) chain_mv<LMAX, NL, L, true>(w.v, G[L - 1], dummy, r[L - 2]);
  if constexpr (L >= 3) chain_mv<LMAX, NL, L - 1, false>(w.v, G[L - 2], r[L - 2], r[L - 3]);
  float rb[kGenMaxD], nb[kGenMaxD], gb[S];
#pragma unroll
  for (int a = 0; a < S; ++a) rb[a] = io.Qb[o + a];
  // k = 1 .. L: Gammabar^k, and rbar_{k+1} for k < L
  auto flush = [&](int k) {
    float* g = io.Gb[k] + o;
#pragma unroll
    for (int b = 0; b < S; ++b) g[b] += gb[b];
  };
  if constexpr (L == 1) {
    chain_adj<LMAX, NL, 1, true, false>(w.v, G[0], rb, dummy, gb, nb);
    flush(1);
  } else {
    chain_adj<LMAX, NL, 1, false, true>(w.v, G[0], rb, r[0], gb, nb);
    flush(1);
    if constexpr (L == 2) {
      chain_adj<LMAX, NL, 2, true, false>(w.v, G[1], nb, dummy, gb, rb);
      flush(2);
    } else {
      chain_adj<LMAX, NL, 2, false, true>(w.v, G[1], nb, r[1], gb, rb);
      flush(2);
      chain_adj<LMAX, NL, 3, true, false>(w.v, G[2], rb, dummy, gb, nb);
      flush(3);
    }
  }
}

// Per edge, once every layer's adjoint is in (after layer 1's chain):
//   w^0bar_{e,u,l} = sum_{a in l} Y_e[a] qs[a],  qs[a] = sum_L sbar^L_{e,u} Q^L[a]
//   wbar^1_{e,u,l} = nu sum_{a in l} Gammabar^1[a] Y_e[a]
//   Ybar_e[a]      = sum_u (w^0_{e,u,l(a)} qs[a] + nu sum_L w^L_{e,u,l(a)} Gammabar^L[a])
// The channel sums of Ybar: warp halving sums, then the warps' partials in a fixed order.
template <typename T, int LMAX, int NL>
__global__ void __launch_bounds__(kMaxChannels) gen_edge_final_kernel(GenRowIO io) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  static_assert(S <= 16, "halving sums of 16 components");
  // per-warp channel partials of Ybar for batches of kEdgeBatch edges, double-buffered:
  // one barrier per batch
  constexpr int kEdgeBatch = 8;
  __shared__ float red[2][kEdgeBatch][kMaxChannels / 32][16];
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na) return;
  const bool act = u < io.C;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = (int)(blockDim.x >> 5);
  float q[NL][S], gb[NL][S];
  const size_t o = ((size_t)ia * io.C + (act ? u : 0)) * S;
#pragma unroll
  for (int L = 0; L < NL; ++L)
#pragma unroll
    for (int a = 0; a < S; ++a) {
      q[L][a] = act ? io.Q[L + 1][o + a] : 0.0f;
      gb[L][a] = act ? io.nu * io.Gb[L + 1][o + a] : 0.0f;
    }
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  T* w0b = reinterpret_cast<T*>(io.wbar[0]);
  T* w1b = reinterpret_cast<T*>(io.wbar[1]);
  float gmax = 0.0f;
  // the batch's sums over the warps, in a fixed order: thread t takes edge t / S, component t % S
  auto flush = [&](int eb, int nb, int buf) {
    for (int t = threadIdx.x; t < nb * S; t += blockDim.x) {
      const int j = t / S, a = t - j * S;
      float sum = 0.0f;
      for (int k = 0; k < nwarp; ++k) sum += red[buf][j][k][a];
      io.Ybar[(size_t)(eb + j) * S + a] = sum;
    }
  };
  for (int e = rb, buf = 0; e < re; ++e) {
    const int j = (e - rb) % kEdgeBatch;
    float y[S];
    load_y<S>(io.Y + (size_t)e * S, y);
    float yc[16];
#pragma unroll
    for (int a = 0; a < 16; ++a) yc[a] = 0.0f;
    if (act) {
      float qs[S], w0l[LM], g0[LM] = {}, g1[LM] = {};
#pragma unroll
      for (int a = 0; a < S; ++a) qs[a] = 0.0f;
#pragma unroll
      for (int L = 0; L < NL; ++L) {
        const float sb = gld(reinterpret_cast<const T*>(io.sbar[L + 1]) + (size_t)e * io.ldsbar[L + 1] +
                             io.sbar_off[L + 1] + u);
        float wl[LM];
        load_lm<T, LM>(reinterpret_cast<const T*>(io.w[L + 1]) + (size_t)e * io.ldw[L + 1] + io.wcol[L + 1] + u * LM,
                       wl);
#pragma unroll
        for (int a = 0; a < S; ++a) {
          qs[a] = fmaf(sb, q[L][a], qs[a]);
          yc[a] = fmaf(wl[l_of(a)], gb[L][a], yc[a]);
        }
      }
      load_lm<T, LM>(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM, w0l);
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const float ya = y[a];
        g0[l_of(a)] = fmaf(ya, qs[a], g0[l_of(a)]);
        g1[l_of(a)] = fmaf(ya, gb[0][a], g1[l_of(a)]);
        yc[a] = fmaf(w0l[l_of(a)], qs[a], yc[a]);
      }
      store_lm<T, LM>(w0b + (size_t)e * io.ldwbar[0] + io.wbcol[0] + u * LM, g0);
      store_lm<T, LM>(w1b + (size_t)e * io.ldwbar[1] + io.wbcol[1] + u * LM, g1);
#pragma unroll
      for (int l = 0; l < LM; ++l) gmax = fmaxf(gmax, fmaxf(fabsf(g0[l]), fabsf(g1[l])));
    }
    const float t = warp_sum16(yc);   // component lane / 2
    if ((lane & 1) == 0) red[buf][j][wid][lane >> 1] = t;
    if (j == kEdgeBatch - 1 || e == re - 1) {
      // one barrier per batch: the other buffer is rewritten only after the next one
      __syncthreads();
      flush(e - j, j + 1, buf);
      buf ^= 1;
    }
  }
  record_amax(io.amax_wbar, gmax);
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Warp-per-atom forms of the per-edge row kernels (environment sums, s, Qbar,
// wbar of the upper layers): one warp owns a centre atom's row, lane t the CPL
// channels t, t + 32, ... (CPL = C / 32, at least 1; lanes past C idle), so
// each per-channel load or store of the warp covers 32 consecutive channels
// (one contiguous span of the edge's row).  A lane's harmonics loads serve all
// its CPL channels.
// ---------------------------------------------------------------------------
constexpr int kGenWarps = 4;   // atoms (warps) per block

struct GenLane {
  int ia, lane, rb, re;
  bool act;
};
template <int CPL>
__device__ __forceinline__ bool gen_lane(const GenRowIO& io, GenLane& g) {
  g.ia = blockIdx.x * kGenWarps + (threadIdx.x >> 5);
  g.lane = threadIdx.x & 31;
  if (g.ia >= io.na) return false;
  g.act = g.lane < io.C;
  g.rb = io.row_ptr[io.a0 + g.ia] - io.e0;
  g.re = io.row_ptr[io.a0 + g.ia + 1] - io.e0;
  return true;
}

// Gamma^L[i][u][b] = nu sum_{e in row i} w^L[e][u][l(b)] Y[e][b]
template <typename T, int LMAX, int CPL>
__global__ void __launch_bounds__(32 * kGenWarps) gen_env_w_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  GenLane g;
  if (!gen_lane<CPL>(io, g) || !g.act) return;
  const T* __restrict__ w = reinterpret_cast<const T*>(io.w[L]) + io.wcol[L] + g.lane * LM;
  const float* __restrict__ Y = io.Y;
  const int ldw = io.ldw[L];
  float G[CPL][S];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int b = 0; b < S; ++b) G[c][b] = 0.0f;
#pragma unroll 2
  for (int e = g.rb; e < g.re; ++e) {
    float y[S];
    load_y<S>(Y + (size_t)e * S, y);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float wl[LM];
      load_lm<T, LM>(w + (size_t)e * ldw + 32 * c * LM, wl);
#pragma unroll
      for (int b = 0; b < S; ++b) G[c][b] = fmaf(wl[l_of(b)], y[b], G[c][b]);
    }
  }
  float* out = io.G[L] + ((size_t)g.ia * io.C + g.lane) * S;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int b = 0; b < S; ++b) out[32 * c * S + b] = G[c][b] * io.nu;
}

// s^L_e[u] = sum_a w^0_{e,u,l(a)} Y_e[a] Q^L[i][u][a], into the s columns of the latent input
template <typename T, int LMAX, int CPL>
__global__ void __launch_bounds__(32 * kGenWarps) gen_s_w_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  GenLane g;
  if (!gen_lane<CPL>(io, g) || !g.act) return;
  const T* __restrict__ w0 = reinterpret_cast<const T*>(io.w[0]) + io.wcol[0] + g.lane * LM;
  const float* __restrict__ Y = io.Y;
  float q[CPL][S];
  const float* Q = io.Q[L] + ((size_t)g.ia * io.C + g.lane) * S;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int a = 0; a < S; ++a) q[c][a] = Q[32 * c * S + a];
  T* __restrict__ xs = reinterpret_cast<T*>(io.xs[L]) + io.xs_off[L] + g.lane;
  const int ldw0 = io.ldw[0], ldxs = io.ldxs[L];
  float smax = 0.0f;
  // the loads of an edge's weights and harmonics are all issued before its stores
#pragma unroll 2
  for (int e = g.rb; e < g.re; ++e) {
    float y[S], wl[CPL][LM];
    load_y<S>(Y + (size_t)e * S, y);
#pragma unroll
    for (int c = 0; c < CPL; ++c) load_lm<T, LM>(w0 + (size_t)e * ldw0 + 32 * c * LM, wl[c]);
    float sv[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      sv[c] = 0.0f;
#pragma unroll
      for (int a = 0; a < S; ++a) sv[c] = fmaf(wl[c][l_of(a)] * y[a], q[c][a], sv[c]);
      smax = fmaxf(smax, fabsf(sv[c]));
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) gst(xs + (size_t)e * ldxs + 32 * c, sv[c]);
  }
  record_amax(io.amax_s, smax);
}

// Qbar^L[i][u][a] = sum_e sbar^L_e[u] w^0_{e,u,l(a)} Y_e[a]
template <typename T, int LMAX, int CPL>
__global__ void __launch_bounds__(32 * kGenWarps) gen_qbar_w_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  GenLane g;
  if (!gen_lane<CPL>(io, g) || !g.act) return;
  const T* __restrict__ w0 = reinterpret_cast<const T*>(io.w[0]) + io.wcol[0] + g.lane * LM;
  const T* __restrict__ sb = reinterpret_cast<const T*>(io.sbar[L]) + io.sbar_off[L] + g.lane;
  const float* __restrict__ Y = io.Y;
  float acc[CPL][S];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int a = 0; a < S; ++a) acc[c][a] = 0.0f;
#pragma unroll 2
  for (int e = g.rb; e < g.re; ++e) {
    float y[S];
    load_y<S>(Y + (size_t)e * S, y);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const float sv = gld(sb + (size_t)e * io.ldsbar[L] + 32 * c);
      float wl[LM];
      load_lm<T, LM>(w0 + (size_t)e * io.ldw[0] + 32 * c * LM, wl);
#pragma unroll
      for (int a = 0; a < S; ++a) acc[c][a] = fmaf(wl[l_of(a)] * sv, y[a], acc[c][a]);
    }
  }
  float* out = io.Qb + ((size_t)g.ia * io.C + g.lane) * S;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int a = 0; a < S; ++a) out[32 * c * S + a] = acc[c][a];
}

// wbar^L_{e,u,l} = nu sum_m Gammabar^L[i][u][lm] Y_e[lm], for a layer L >= 2
template <typename T, int LMAX, int CPL>
__global__ void __launch_bounds__(32 * kGenWarps) gen_wbar_w_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  GenLane g;
  if (!gen_lane<CPL>(io, g) || !g.act) return;
  float gb[CPL][S];
  const float* G = io.Gb[L] + ((size_t)g.ia * io.C + g.lane) * S;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int a = 0; a < S; ++a) gb[c][a] = io.nu * G[32 * c * S + a];
  T* __restrict__ wLb = reinterpret_cast<T*>(io.wbar[L]) + io.wbcol[L] + g.lane * LM;
  const float* __restrict__ Y = io.Y;
  float gmax = 0.0f;
#pragma unroll 2
  for (int e = g.rb; e < g.re; ++e) {
    float y[S];
    load_y<S>(Y + (size_t)e * S, y);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float o[LM] = {};
#pragma unroll
      for (int a = 0; a < S; ++a) o[l_of(a)] = fmaf(gb[c][a], y[a], o[l_of(a)]);
#pragma unroll
      for (int l = 0; l < LM; ++l) gmax = fmaxf(gmax, fabsf(o[l]));
      store_lm<T, LM>(wLb + (size_t)e * io.ldwbar[L] + 32 * c * LM, o);
    }
  }
  record_amax(io.amax_wbar, gmax);
}

static int block_of(int C) { return (C + 31) / 32 * 32; }

// the warp-per-atom kernels at CPL = C / 32 channels per lane (C a power of two, 8..128)
#define GEN_W_LAUNCH(KERNEL, ...)                                                     \
  do {                                                                                \
    const dim3 grid_((io.na + kGenWarps - 1) / kGenWarps), block_(32 * kGenWarps);    \
    if (io.C >= 128) KERNEL<T, LMAX, 4><<<grid_, block_, 0, st>>>(__VA_ARGS__);       \
    else if (io.C >= 64) KERNEL<T, LMAX, 2><<<grid_, block_, 0, st>>>(__VA_ARGS__);   \
    else KERNEL<T, LMAX, 1><<<grid_, block_, 0, st>>>(__VA_ARGS__);                   \
  } while (0)

template <int LMAX, int NL>
static GenVals<LMAX, NL> vals_of(const GenRowIO& io) {
  GenVals<LMAX, NL> w;
  for (int q = 0; q < GenVals<LMAX, NL>::n; ++q) w.v[q] = io.vals[q];
  return w;
}

template <int LMAX, int NL>
static void chain_fwd(const GenRowIO& io, int L, cudaStream_t st) {
  const GenVals<LMAX, NL> w = vals_of<LMAX, NL>(io);
  const int g = (io.na * io.C + kChainThreads - 1) / kChainThreads;
  if (L == 1) gen_chain_fwd_kernel<LMAX, NL, 1><<<g, kChainThreads, 0, st>>>(io, w);
  if constexpr (NL >= 2) if (L == 2) gen_chain_fwd_kernel<LMAX, NL, 2><<<g, kChainThreads, 0, st>>>(io, w);
  if constexpr (NL >= 3) if (L == 3) gen_chain_fwd_kernel<LMAX, NL, 3><<<g, kChainThreads, 0, st>>>(io, w);
}

template <int LMAX, int NL>
static void chain_bwd(const GenRowIO& io, int L, cudaStream_t st) {
  const GenVals<LMAX, NL> w = vals_of<LMAX, NL>(io);
  const int g = (io.na * io.C + kChainThreads - 1) / kChainThreads;
  if (L == 1) gen_chain_bwd_kernel<LMAX, NL, 1><<<g, kChainThreads, 0, st>>>(io, w);
  if constexpr (NL >= 2) if (L == 2) gen_chain_bwd_kernel<LMAX, NL, 2><<<g, kChainThreads, 0, st>>>(io, w);
  if constexpr (NL >= 3) if (L == 3) gen_chain_bwd_kernel<LMAX, NL, 3><<<g, kChainThreads, 0, st>>>(io, w);
}

// the (l_max, layers) models of the generic path
template <int LMAX>
static void chain_fwd_nl(const GenRowIO& io, int L, cudaStream_t st) {
  if (io.nl == 1) chain_fwd<LMAX, 1>(io, L, st);
  else if (io.nl == 2) chain_fwd<LMAX, 2>(io, L, st);
  else chain_fwd<LMAX, 3>(io, L, st);
}
template <int LMAX>
static void chain_bwd_nl(const GenRowIO& io, int L, cudaStream_t st) {
  if (io.nl == 1) chain_bwd<LMAX, 1>(io, L, st);
  else if (io.nl == 2) chain_bwd<LMAX, 2>(io, L, st);
  else chain_bwd<LMAX, 3>(io, L, st);
}

template <typename T, int LMAX>
static void fwd_lmax(const GenRowIO& io, int L, cudaStream_t st) {
  GEN_W_LAUNCH(gen_env_w_kernel, io, L);
  chain_fwd_nl<LMAX>(io, L, st);
  GEN_W_LAUNCH(gen_s_w_kernel, io, L);
}

template <typename T, int LMAX>
static void bwd_lmax(const GenRowIO& io, int L, cudaStream_t st) {
  const int bl = block_of(io.C);
  if (L == io.nl) {
    for (int k = 1; k <= io.nl; ++k)
      cudaMemsetAsync(io.Gb[k], 0, (size_t)io.na * io.C * io.S * sizeof(float), st);
  }
  GEN_W_LAUNCH(gen_qbar_w_kernel, io, L);
  chain_bwd_nl<LMAX>(io, L, st);
  if (L >= 2) GEN_W_LAUNCH(gen_wbar_w_kernel, io, L);
  else if (io.nl == 1) gen_edge_final_kernel<T, LMAX, 1><<<io.na, bl, 0, st>>>(io);
  else if (io.nl == 2) gen_edge_final_kernel<T, LMAX, 2><<<io.na, bl, 0, st>>>(io);
  else gen_edge_final_kernel<T, LMAX, 3><<<io.na, bl, 0, st>>>(io);
}

template <typename T>
void gen_row_fwd(const GenRowIO& io, int L, cudaStream_t st) {
  if (io.na <= 0) return;
  if (io.lmax == 1) fwd_lmax<T, 1>(io, L, st);
  else if (io.lmax == 2) fwd_lmax<T, 2>(io, L, st);
  else fwd_lmax<T, 3>(io, L, st);
}

template <typename T>
void gen_row_bwd(const GenRowIO& io, int L, cudaStream_t st) {
  if (io.na <= 0) return;
  if (io.lmax == 1) bwd_lmax<T, 1>(io, L, st);
  else if (io.lmax == 2) bwd_lmax<T, 2>(io, L, st);
  else bwd_lmax<T, 3>(io, L, st);
}

template <int LMAX, int NL, int K>
static void pack_layer(const std::vector<double>& W, int S, std::vector<float>& vals, std::vector<char>& hit) {
  using P = Cand<LMAX, NL, K>;
  for (int q = 0; q < P::n; ++q) {
    const size_t i = ((size_t)P::list.a[q] * S + P::list.b[q]) * P::dout + P::list.c[q];
    vals.push_back((float)W[i]);
    hit[i] = 1;
  }
}

template <int LMAX, int NL>
static bool pack_model(const std::vector<std::vector<Irrep>>& irs, const std::vector<std::vector<double>>& W,
                       std::vector<float>& vals, std::string& why) {
  constexpr int S = (LMAX + 1) * (LMAX + 1);
  vals.clear();
  for (int K = 0; K <= NL; ++K) {   // the compile-time irreps are the model's
    const IrSet ct = ir_layer(LMAX, NL, K);
    bool same = ct.n == (int)irs[K].size();
    for (int q = 0; same && q < ct.n; ++q) same = ct.l[q] == irs[K][q].l && ct.p[q] == irs[K][q].p;
    if (!same) {
      why = "layer " + std::to_string(K) + " irreps differ from the generic kernels'";
      return false;
    }
  }
  for (int K = 1; K <= NL; ++K) {
    std::vector<char> hit(W[K].size(), 0);
    if (K == 1) pack_layer<LMAX, NL, 1>(W[K], S, vals, hit);
    if constexpr (NL >= 2) if (K == 2) pack_layer<LMAX, NL, 2>(W[K], S, vals, hit);
    if constexpr (NL >= 3) if (K == 3) pack_layer<LMAX, NL, 3>(W[K], S, vals, hit);
    double wmax = 0.0, missed = 0.0;
    for (size_t i = 0; i < W[K].size(); ++i) {
      wmax = std::fmax(wmax, std::fabs(W[K][i]));
      if (!hit[i]) missed = std::fmax(missed, std::fabs(W[K][i]));
    }
    if (missed > 1e-12 * wmax) {
      why = "layer " + std::to_string(K) + " tensor has a nonzero outside the candidate pattern";
      return false;
    }
  }
  return (int)vals.size() == GenVals<LMAX, NL>::n;
}

bool gen_pack_values(int lmax, int nl, const std::vector<std::vector<Irrep>>& irs,
                     const std::vector<std::vector<double>>& W, std::vector<float>& vals, std::string& why) {
  if ((int)irs.size() != nl + 1 || (int)W.size() != nl + 1) {
    why = "layer count mismatch";
    return false;
  }
  const int code = lmax * 10 + nl;
  switch (code) {
    case 11: return pack_model<1, 1>(irs, W, vals, why);
    case 12: return pack_model<1, 2>(irs, W, vals, why);
    case 13: return pack_model<1, 3>(irs, W, vals, why);
    case 21: return pack_model<2, 1>(irs, W, vals, why);
    case 22: return pack_model<2, 2>(irs, W, vals, why);
    case 23: return pack_model<2, 3>(irs, W, vals, why);
    case 31: return pack_model<3, 1>(irs, W, vals, why);
    case 32: return pack_model<3, 2>(irs, W, vals, why);
    case 33: return pack_model<3, 3>(irs, W, vals, why);
    default: why = "l_max " + std::to_string(lmax) + ", " + std::to_string(nl) + " layers: not supported"; return false;
  }
}

template void gen_row_fwd<float>(const GenRowIO&, int, cudaStream_t);
template void gen_row_fwd<bf16>(const GenRowIO&, int, cudaStream_t);
template void gen_row_bwd<float>(const GenRowIO&, int, cudaStream_t);
template void gen_row_bwd<bf16>(const GenRowIO&, int, cudaStream_t);

}  // namespace alg
