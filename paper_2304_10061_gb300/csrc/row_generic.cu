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
//   w^0bar_{e,l} += sum_{a in l} sbar^L_e Y_e[a] Q^L[a]
//   Ybar_e[a]    += sum_u (sbar^L_e w^0_{e,l(a)} Q^L[a] + nu w^L_{e,l(a)} Gammabar^L[a])
// processed for L = nl, nl-1, ..., 1 (the order in which the sbar^L arrive):
// Gammabar^L is complete once every layer >= L has been processed.
//
// Layout: per atom [atom][channel][S] float32; per edge the activation-type
// arrays of the MLP side (w, s, sbar, wbar) and float32 Y / Ybar / w^0bar.
// Row kernels: one block per centre atom, one thread per channel; per-atom
// sums are register accumulations over the row (deterministic), the channel
// sums of Ybar are block reductions in a fixed order; l_max is a template
// parameter, so every per-edge vector lives in registers.  Chain kernels: one
// thread per (atom, channel); every thread's vectors in shared memory
// ([component][thread], conflict-free); the nonzero lists (read by all threads
// alike, so broadcast from L1) sorted by the output index of each sum, the
// running sum in a register.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

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

// Sum of v over the block's threads (blockDim.x a multiple of 32, <= 1024), the
// same fixed order every time; red: 32 floats of shared memory.
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float t = 0.0f;
  for (int q = 0; q < nw; ++q) t += red[q];
  return t;
}

constexpr int kChainThreads = 64;   // (atom, channel) pairs per block of the chain kernels

// A thread's vectors in shared memory, [component][thread] (conflict-free):
// `ng` slots of S components (the environments Gamma^k) first, then slots of
// D components (the largest feature dimension of the model).
struct Vecs {
  float* base;
  int tid, S, ng, D;
  __device__ __forceinline__ float& at(int slot, int i) const {
    const int off = slot < ng ? slot * S : ng * S + (slot - ng) * D;
    return base[(size_t)(off + i) * kChainThreads + tid];
  }
};

// sum over the entries of a nonzero list sorted by its `key` component, flushed per key
// run: out(key, sum of term(entry)) once per distinct key, in list order
template <typename Key, typename Term, typename Out>
__device__ __forceinline__ void sorted_sum(const GenNz* z, int n, Key&& key, Term&& term, Out&& out) {
  int run = -1;
  float acc = 0.0f;
  for (int q = 0; q < n; ++q) {
    const GenNz zz = z[q];
    const int k = key(zz);
    if (k != run) {
      if (run >= 0) out(run, acc);
      run = k;
      acc = 0.0f;
    }
    acc += term(zz);
  }
  if (run >= 0) out(run, acc);
}

}  // namespace

// Gamma^L[i][u][b] = nu sum_{e in row i} w^L[e][u][l(b)] Y[e][b]
template <typename T, int LMAX>
__global__ void gen_env_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na || u >= io.C) return;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w = reinterpret_cast<const T*>(io.w[L]);
  const int ldw = io.ldw[L], col = io.wcol[L];
  float G[S];
#pragma unroll
  for (int b = 0; b < S; ++b) G[b] = 0.0f;
  for (int e = rb; e < re; ++e) {
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = gld(w + (size_t)e * ldw + col + u * LM + l);
    const float* y = io.Y + (size_t)e * S;
#pragma unroll
    for (int b = 0; b < S; ++b) G[b] += wl[l_of(b)] * y[b];
  }
  float* out = io.G[L] + ((size_t)ia * io.C + u) * S;
#pragma unroll
  for (int b = 0; b < S; ++b) out[b] = G[b] * io.nu;
}

// Q^L[i][u][:] = M^1 ... M^L e_0
__global__ void __launch_bounds__(kChainThreads) gen_chain_fwd_kernel(GenRowIO io, int L) {
  extern __shared__ __align__(16) float sm[];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= io.na * io.C) return;
  const int ia = t / io.C, u = t - ia * io.C;
  const size_t o = ((size_t)ia * io.C + u) * io.S;
  // slots: Gamma^1..Gamma^L (S each), then the two chain vectors
  const Vecs V{sm, (int)threadIdx.x, io.S, L, io.dmax};
  for (int k = 1; k <= L; ++k)
    for (int b = 0; b < io.S; ++b) V.at(k - 1, b) = io.G[k][o + b];
  int cur = L, nxt = L + 1;
  for (int k = L; k >= 1; --k) {   // r <- M^k r; the first step acts on e_0 (its c == 0 entries)
    const bool first = (k == L);
    for (int a = 0; a < io.dim[k - 1]; ++a) V.at(nxt, a) = 0.0f;
    sorted_sum(first ? io.nz0[k] : io.nz[k], first ? io.nnz0[k] : io.nnz[k], [](const GenNz& z) { return (int)z.a; },
               [&](const GenNz& z) { return z.v * V.at(k - 1, z.b) * (first ? 1.0f : V.at(cur, z.c)); },
               [&](int a, float v) { V.at(nxt, a) = v; });
    const int sw = cur; cur = nxt; nxt = sw;
  }
  float* q = io.Q[L] + o;
  for (int a = 0; a < io.S; ++a) q[a] = V.at(cur, a);
}

// s^L_e[u] = sum_a w^0_{e,u,l(a)} Y_e[a] Q^L[i][u][a], into the s columns of the latent input
template <typename T, int LMAX>
__global__ void gen_s_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na || u >= io.C) return;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  float q[S];
  const float* Q = io.Q[L] + ((size_t)ia * io.C + u) * S;
#pragma unroll
  for (int a = 0; a < S; ++a) q[a] = Q[a];
  T* xs = reinterpret_cast<T*>(io.xs[L]);
  for (int e = rb; e < re; ++e) {
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = gld(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM + l);
    const float* y = io.Y + (size_t)e * S;
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < S; ++a) s += wl[l_of(a)] * y[a] * q[a];
    gst(xs + (size_t)e * io.ldxs[L] + io.xs_off[L] + u, s);
  }
}

// Qbar^L[i][u][a] = sum_e sbar^L_e[u] w^0_{e,u,l(a)} Y_e[a]
template <typename T, int LMAX>
__global__ void gen_qbar_kernel(GenRowIO io, int L) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na || u >= io.C) return;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  const T* sb = reinterpret_cast<const T*>(io.sbar[L]);
  float acc[S];
#pragma unroll
  for (int a = 0; a < S; ++a) acc[a] = 0.0f;
  for (int e = rb; e < re; ++e) {
    const float s = gld(sb + (size_t)e * io.ldsbar[L] + io.sbar_off[L] + u);
    float wl[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) wl[l] = s * gld(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM + l);
    const float* y = io.Y + (size_t)e * S;
#pragma unroll
    for (int a = 0; a < S; ++a) acc[a] += wl[l_of(a)] * y[a];
  }
  float* out = io.Qb + ((size_t)ia * io.C + u) * S;
#pragma unroll
  for (int a = 0; a < S; ++a) out[a] = acc[a];
}

// Back along the chain of Q^L: Gammabar^k += ..., k = 1..L.  Each sum runs over
// a copy of the layer's nonzeros sorted by its output index (a, b or c), so it
// accumulates in a register and is written once.
__global__ void __launch_bounds__(kChainThreads) gen_chain_bwd_kernel(GenRowIO io, int L) {
  extern __shared__ __align__(16) float sm[];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= io.na * io.C) return;
  const int ia = t / io.C, u = t - ia * io.C;
  const size_t o = ((size_t)ia * io.C + u) * io.S;
  // slots: Gamma^1..Gamma^L (S each); r_k at slot L - 2 + k for k = 2..L + 1; rbar; nbar
  const Vecs V{sm, (int)threadIdx.x, io.S, L, io.dmax};
  auto sR = [&](int k) { return L - 2 + k; };
  const int sRb = 2 * L, sNb = 2 * L + 1;
  for (int k = 1; k <= L; ++k)
    for (int b = 0; b < io.S; ++b) V.at(k - 1, b) = io.G[k][o + b];
  // r_{L+1} = e_0; r_k = M^k r_{k+1} for k = L .. 2
  for (int c = 0; c < io.dim[L]; ++c) V.at(sR(L + 1), c) = 0.0f;
  V.at(sR(L + 1), 0) = 1.0f;
  for (int k = L; k >= 2; --k) {   // r_{L+1} = e_0: the first step takes the c == 0 entries
    for (int a = 0; a < io.dim[k - 1]; ++a) V.at(sR(k), a) = 0.0f;
    sorted_sum(k == L ? io.nz0[k] : io.nz[k], k == L ? io.nnz0[k] : io.nnz[k], [](const GenNz& z) { return (int)z.a; },
               [&](const GenNz& z) { return z.v * V.at(k - 1, z.b) * V.at(sR(k + 1), z.c); },
               [&](int a, float v) { V.at(sR(k), a) = v; });
  }
  // rbar_1 = Qbar^L; for k = 1..L: Gammabar^k[b] += W rbar_k[a] r_{k+1}[c], rbar_{k+1}[c] = W rbar_k[a] Gamma^k[b]
  for (int a = 0; a < io.S; ++a) V.at(sRb, a) = io.Qb[o + a];
  for (int k = 1; k <= L; ++k) {
    float* Gb = io.Gb[k] + o;
    sorted_sum(k == L ? io.nz0b[k] : io.nzb[k], k == L ? io.nnz0[k] : io.nnz[k], [](const GenNz& z) { return (int)z.b; },
               [&](const GenNz& z) { return z.v * V.at(sRb, z.a) * V.at(sR(k + 1), z.c); },
               [&](int b, float v) { Gb[b] += v; });
    if (k < L) {
      for (int c = 0; c < io.dim[k]; ++c) V.at(sNb, c) = 0.0f;
      sorted_sum(io.nzc[k], io.nnz[k], [](const GenNz& z) { return (int)z.c; },
                 [&](const GenNz& z) { return z.v * V.at(sRb, z.a) * V.at(k - 1, z.b); },
                 [&](int c, float v) { V.at(sNb, c) = v; });
      for (int c = 0; c < io.dim[k]; ++c) V.at(sRb, c) = V.at(sNb, c);
    }
  }
}

// Per edge, layer L: wbar^L, the w^0bar accumulation and the Ybar accumulation.
// last = true (L == 1): w^0bar is complete; written to its activation-type slot.
template <typename T, int LMAX>
__global__ void gen_edge_adj_kernel(GenRowIO io, int L, bool last) {
  constexpr int S = (LMAX + 1) * (LMAX + 1), LM = LMAX + 1;
  __shared__ float red[(kMaxChannels / 32) * 16];
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na) return;
  const bool act = u < io.C;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  const T* wL = reinterpret_cast<const T*>(io.w[L]);
  const T* sb = reinterpret_cast<const T*>(io.sbar[L]);
  T* wLb = reinterpret_cast<T*>(io.wbar[L]);
  T* w0b = reinterpret_cast<T*>(io.wbar[0]);
  float q[S], gbar[S];
  const size_t o = ((size_t)ia * io.C + (act ? u : 0)) * S;
#pragma unroll
  for (int a = 0; a < S; ++a) {
    q[a] = act ? io.Q[L][o + a] : 0.0f;
    gbar[a] = act ? io.Gb[L][o + a] : 0.0f;
  }
  for (int e = rb; e < re; ++e) {
    const float* y = io.Y + (size_t)e * S;
    float yv[S], yc[S];
#pragma unroll
    for (int a = 0; a < S; ++a) {
      yv[a] = y[a];
      yc[a] = 0.0f;
    }
    if (act) {
      const float s = gld(sb + (size_t)e * io.ldsbar[L] + io.sbar_off[L] + u);
      float w0l[LM], wLl[LM], g0[LM], gL[LM];
#pragma unroll
      for (int l = 0; l < LM; ++l) {
        w0l[l] = gld(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM + l);
        wLl[l] = gld(wL + (size_t)e * io.ldw[L] + io.wcol[L] + u * LM + l);
        g0[l] = 0.0f;
        gL[l] = 0.0f;
      }
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const int l = l_of(a);
        g0[l] += s * yv[a] * q[a];
        gL[l] += io.nu * gbar[a] * yv[a];
        yc[a] = s * w0l[l] * q[a] + io.nu * wLl[l] * gbar[a];
      }
      float* acc = io.w0bar + ((size_t)e * io.C + u) * LM;
#pragma unroll
      for (int l = 0; l < LM; ++l) {
        const float t = (L == io.nl ? 0.0f : acc[l]) + g0[l];
        if (last) gst(w0b + (size_t)e * io.ldwbar[0] + io.wbcol[0] + u * LM + l, t);
        else acc[l] = t;
        gst(wLb + (size_t)e * io.ldwbar[L] + io.wbcol[L] + u * LM + l, gL[l]);
      }
    }
    // channel sums of the S components: warp shuffles, then the warps' partials in a fixed order
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) yc[a] += __shfl_xor_sync(0xffffffffu, yc[a], o2);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int a = 0; a < S; ++a) red[(threadIdx.x >> 5) * S + a] = yc[a];
    __syncthreads();
    if (threadIdx.x < S) {
      float t = 0.0f;
      for (int q2 = 0; q2 < (int)(blockDim.x >> 5); ++q2) t += red[q2 * S + threadIdx.x];
      float* yb = io.Ybar + (size_t)e * S + threadIdx.x;
      *yb = (L == io.nl ? 0.0f : *yb) + t;
    }
  }
}

// ---------------------------------------------------------------------------
static int block_of(int C) { return (C + 31) / 32 * 32; }

// shared memory of a chain kernel: L environment slots of S components and nslot of dmax per thread
static size_t chain_smem(const GenRowIO& io, int L, int nslot) {
  return ((size_t)L * io.S + (size_t)nslot * io.dmax) * kChainThreads * sizeof(float);
}

// the chain kernels' opt-in to large dynamic shared memory, once per device
static void chain_smem_opt_in() {
  static bool done[64] = {};
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= 64 || done[d]) return;
  cudaFuncSetAttribute(gen_chain_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(gen_chain_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  done[d] = true;
}

template <typename T, int LMAX>
static void fwd_lmax(const GenRowIO& io, int L, cudaStream_t st) {
  const int bl = block_of(io.C);
  gen_env_kernel<T, LMAX><<<io.na, bl, 0, st>>>(io, L);
  const int n = io.na * io.C;
  const size_t sm = chain_smem(io, L, 2);
  chain_smem_opt_in();
  gen_chain_fwd_kernel<<<(n + kChainThreads - 1) / kChainThreads, kChainThreads, sm, st>>>(io, L);
  gen_s_kernel<T, LMAX><<<io.na, bl, 0, st>>>(io, L);
}

template <typename T, int LMAX>
static void bwd_lmax(const GenRowIO& io, int L, cudaStream_t st) {
  const int bl = block_of(io.C);
  if (L == io.nl) {
    for (int k = 1; k <= io.nl; ++k)
      cudaMemsetAsync(io.Gb[k], 0, (size_t)io.na * io.C * io.S * sizeof(float), st);
  }
  gen_qbar_kernel<T, LMAX><<<io.na, bl, 0, st>>>(io, L);
  const int n = io.na * io.C;
  const size_t sm = chain_smem(io, L, L + 2);
  chain_smem_opt_in();
  gen_chain_bwd_kernel<<<(n + kChainThreads - 1) / kChainThreads, kChainThreads, sm, st>>>(io, L);
  gen_edge_adj_kernel<T, LMAX><<<io.na, bl, 0, st>>>(io, L, L == 1);
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

template void gen_row_fwd<float>(const GenRowIO&, int, cudaStream_t);
template void gen_row_fwd<bf16>(const GenRowIO&, int, cudaStream_t);
template void gen_row_bwd<float>(const GenRowIO&, int, cudaStream_t);
template void gen_row_bwd<bf16>(const GenRowIO&, int, cudaStream_t);

}  // namespace alg
