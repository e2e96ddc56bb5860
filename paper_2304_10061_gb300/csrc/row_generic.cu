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
// One block per centre atom, one thread per channel: per-atom sums are
// register accumulations over the row (deterministic), the channel sums of
// Ybar are block reductions in a fixed order.
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

__device__ __forceinline__ int l_of(int a) { return a < 1 ? 0 : (a < 4 ? 1 : (a < 9 ? 2 : 3)); }

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

}  // namespace

// Gamma^L[i][u][b] = nu sum_{e in row i} w^L[e][u][l(b)] Y[e][b]
template <typename T>
__global__ void gen_env_kernel(GenRowIO io, int L) {
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na || u >= io.C) return;
  const int S = io.S, LM = io.lmax + 1;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w = reinterpret_cast<const T*>(io.w[L]);
  const int ldw = io.ldw[L], col = io.wcol[L];
  float G[16];
  for (int b = 0; b < S; ++b) G[b] = 0.0f;
  for (int e = rb; e < re; ++e) {
    float wl[4];
    for (int l = 0; l < LM; ++l) wl[l] = gld(w + (size_t)e * ldw + col + u * LM + l);
    const float* y = io.Y + (size_t)e * S;
    for (int b = 0; b < S; ++b) G[b] += wl[l_of(b)] * y[b];
  }
  float* out = io.G[L] + ((size_t)ia * io.C + u) * S;
  for (int b = 0; b < S; ++b) out[b] = G[b] * io.nu;
}

// The chain r <- M^k r from k = L down to 1, starting from e_0 of V^L's layout.
// Returns r (length S) in `r`; scratch: two vectors of kGenMaxD.
__device__ __forceinline__ void gen_chain(const GenRowIO& io, int ia, int u, int L, float* r, float* t) {
  for (int c = 0; c < io.dim[L]; ++c) r[c] = 0.0f;
  r[0] = 1.0f;
  for (int k = L; k >= 1; --k) {
    const float* G = io.G[k] + ((size_t)ia * io.C + u) * io.S;
    for (int a = 0; a < io.dim[k - 1]; ++a) t[a] = 0.0f;
    const GenNz* nz = io.nz[k];
    for (int q = 0; q < io.nnz[k]; ++q) {
      const GenNz z = nz[q];
      t[z.a] += z.v * G[z.b] * r[z.c];
    }
    for (int a = 0; a < io.dim[k - 1]; ++a) r[a] = t[a];
  }
}

// Q^L[i][u][:] = M^1 ... M^L e_0
__global__ void gen_chain_fwd_kernel(GenRowIO io, int L) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= io.na * io.C) return;
  const int ia = t / io.C, u = t - ia * io.C;
  float r[kGenMaxD], s[kGenMaxD];
  gen_chain(io, ia, u, L, r, s);
  float* q = io.Q[L] + ((size_t)ia * io.C + u) * io.S;
  for (int a = 0; a < io.S; ++a) q[a] = r[a];
}

// s^L_e[u] = sum_a w^0_{e,u,l(a)} Y_e[a] Q^L[i][u][a], into the s columns of the latent input
template <typename T>
__global__ void gen_s_kernel(GenRowIO io, int L) {
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na || u >= io.C) return;
  const int S = io.S, LM = io.lmax + 1;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  float q[16];
  const float* Q = io.Q[L] + ((size_t)ia * io.C + u) * S;
  for (int a = 0; a < S; ++a) q[a] = Q[a];
  T* xs = reinterpret_cast<T*>(io.xs[L]);
  for (int e = rb; e < re; ++e) {
    float wl[4];
    for (int l = 0; l < LM; ++l) wl[l] = gld(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM + l);
    const float* y = io.Y + (size_t)e * S;
    float s = 0.0f;
    for (int a = 0; a < S; ++a) s += wl[l_of(a)] * y[a] * q[a];
    gst(xs + (size_t)e * io.ldxs[L] + io.xs_off[L] + u, s);
  }
}

// Qbar^L[i][u][a] = sum_e sbar^L_e[u] w^0_{e,u,l(a)} Y_e[a]
template <typename T>
__global__ void gen_qbar_kernel(GenRowIO io, int L) {
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na || u >= io.C) return;
  const int S = io.S, LM = io.lmax + 1;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  const T* sb = reinterpret_cast<const T*>(io.sbar[L]);
  float acc[16];
  for (int a = 0; a < S; ++a) acc[a] = 0.0f;
  for (int e = rb; e < re; ++e) {
    const float s = gld(sb + (size_t)e * io.ldsbar[L] + io.sbar_off[L] + u);
    float wl[4];
    for (int l = 0; l < LM; ++l) wl[l] = s * gld(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM + l);
    const float* y = io.Y + (size_t)e * S;
    for (int a = 0; a < S; ++a) acc[a] += wl[l_of(a)] * y[a];
  }
  float* out = io.Qb + ((size_t)ia * io.C + u) * S;
  for (int a = 0; a < S; ++a) out[a] = acc[a];
}

// Back along the chain of Q^L: Gammabar^k += ..., k = 1..L
__global__ void gen_chain_bwd_kernel(GenRowIO io, int L) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= io.na * io.C) return;
  const int ia = t / io.C, u = t - ia * io.C;
  const size_t o = ((size_t)ia * io.C + u) * io.S;
  // R[k] = r_k = M^k ... M^L e_0 for k = L + 1 (e_0) down to 2, kept for the backward sweep
  float R[kGenMaxLayers + 2][kGenMaxD];
  for (int c = 0; c < io.dim[L]; ++c) R[L + 1][c] = 0.0f;
  R[L + 1][0] = 1.0f;
  for (int k = L; k >= 2; --k) {
    const float* G = io.G[k] + o;
    for (int a = 0; a < io.dim[k - 1]; ++a) R[k][a] = 0.0f;
    for (int q = 0; q < io.nnz[k]; ++q) {
      const GenNz z = io.nz[k][q];
      R[k][z.a] += z.v * G[z.b] * R[k + 1][z.c];
    }
  }
  // rbar_1 = Qbar^L; for k = 1..L: Gammabar^k[b] += sum W rbar_k[a] r_{k+1}[c],
  // rbar_{k+1}[c] = sum W rbar_k[a] Gamma^k[b]
  float rb[kGenMaxD], nb[kGenMaxD];
  for (int a = 0; a < io.S; ++a) rb[a] = io.Qb[o + a];
  for (int k = 1; k <= L; ++k) {
    const float* G = io.G[k] + o;
    float gb[16];
    for (int b = 0; b < io.S; ++b) gb[b] = 0.0f;
    for (int c = 0; c < io.dim[k]; ++c) nb[c] = 0.0f;
    for (int q = 0; q < io.nnz[k]; ++q) {
      const GenNz z = io.nz[k][q];
      gb[z.b] += z.v * rb[z.a] * R[k + 1][z.c];
      nb[z.c] += z.v * rb[z.a] * G[z.b];
    }
    float* Gb = io.Gb[k] + o;
    for (int b = 0; b < io.S; ++b) Gb[b] += gb[b];
    for (int c = 0; c < io.dim[k]; ++c) rb[c] = nb[c];
  }
}

// Per edge, layer L: wbar^L, the w^0bar accumulation and the Ybar accumulation.
// last = true (L == 1): w^0bar is complete; written to its activation-type slot.
template <typename T>
__global__ void gen_edge_adj_kernel(GenRowIO io, int L, bool last) {
  __shared__ float red[32];
  const int ia = blockIdx.x, u = threadIdx.x;
  if (ia >= io.na) return;
  const bool act = u < io.C;
  const int S = io.S, LM = io.lmax + 1;
  const int rb = io.row_ptr[io.a0 + ia] - io.e0, re = io.row_ptr[io.a0 + ia + 1] - io.e0;
  const T* w0 = reinterpret_cast<const T*>(io.w[0]);
  const T* wL = reinterpret_cast<const T*>(io.w[L]);
  const T* sb = reinterpret_cast<const T*>(io.sbar[L]);
  T* wLb = reinterpret_cast<T*>(io.wbar[L]);
  T* w0b = reinterpret_cast<T*>(io.wbar[0]);
  float q[16], gbar[16];
  const size_t o = ((size_t)ia * io.C + (act ? u : 0)) * S;
  for (int a = 0; a < S; ++a) {
    q[a] = act ? io.Q[L][o + a] : 0.0f;
    gbar[a] = act ? io.Gb[L][o + a] : 0.0f;
  }
  for (int e = rb; e < re; ++e) {
    const float* y = io.Y + (size_t)e * S;
    float yc[16];
    for (int a = 0; a < S; ++a) yc[a] = 0.0f;
    if (act) {
      const float s = gld(sb + (size_t)e * io.ldsbar[L] + io.sbar_off[L] + u);
      float w0l[4], wLl[4], g0[4], gL[4];
      for (int l = 0; l < LM; ++l) {
        w0l[l] = gld(w0 + (size_t)e * io.ldw[0] + io.wcol[0] + u * LM + l);
        wLl[l] = gld(wL + (size_t)e * io.ldw[L] + io.wcol[L] + u * LM + l);
        g0[l] = 0.0f;
        gL[l] = 0.0f;
      }
      for (int a = 0; a < S; ++a) {
        const int l = l_of(a);
        g0[l] += s * y[a] * q[a];
        gL[l] += io.nu * gbar[a] * y[a];
        yc[a] = s * w0l[l] * q[a] + io.nu * wLl[l] * gbar[a];
      }
      float* acc = io.w0bar + (size_t)e * io.C * LM + u * LM;
      for (int l = 0; l < LM; ++l) {
        const float t = (L == io.nl ? 0.0f : acc[l]) + g0[l];
        if (last) gst(w0b + (size_t)e * io.ldwbar[0] + io.wbcol[0] + u * LM + l, t);
        else acc[l] = t;
        gst(wLb + (size_t)e * io.ldwbar[L] + io.wbcol[L] + u * LM + l, gL[l]);
      }
    }
    for (int a = 0; a < S; ++a) {
      const float t = block_sum(yc[a], red);
      if (threadIdx.x == 0) io.Ybar[(size_t)e * S + a] = (L == io.nl ? 0.0f : io.Ybar[(size_t)e * S + a]) + t;
    }
  }
}

// ---------------------------------------------------------------------------
static int block_of(int C) { return (C + 31) / 32 * 32; }

template <typename T>
void gen_row_fwd(const GenRowIO& io, int L, cudaStream_t st) {
  if (io.na <= 0) return;
  const int bl = block_of(io.C);
  gen_env_kernel<T><<<io.na, bl, 0, st>>>(io, L);
  const int n = io.na * io.C;
  gen_chain_fwd_kernel<<<(n + 127) / 128, 128, 0, st>>>(io, L);
  gen_s_kernel<T><<<io.na, bl, 0, st>>>(io, L);
}

template <typename T>
void gen_row_bwd(const GenRowIO& io, int L, cudaStream_t st) {
  if (io.na <= 0) return;
  const int bl = block_of(io.C);
  if (L == io.nl) {
    for (int k = 1; k <= io.nl; ++k)
      cudaMemsetAsync(io.Gb[k], 0, (size_t)io.na * io.C * io.S * sizeof(float), st);
  }
  gen_qbar_kernel<T><<<io.na, bl, 0, st>>>(io, L);
  const int n = io.na * io.C;
  gen_chain_bwd_kernel<<<(n + 127) / 128, 128, 0, st>>>(io, L);
  gen_edge_adj_kernel<T><<<io.na, bl, 0, st>>>(io, L, L == 1);
}

template void gen_row_fwd<float>(const GenRowIO&, int, cudaStream_t);
template void gen_row_fwd<bf16>(const GenRowIO&, int, cudaStream_t);
template void gen_row_bwd<float>(const GenRowIO&, int, cudaStream_t);
template void gen_row_bwd<bf16>(const GenRowIO&, int, cudaStream_t);

}  // namespace alg
