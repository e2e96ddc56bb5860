// Float32 GEMM on the CUDA cores (the all-float32 path of the MLPs):
//   C[M x N] = A[M x K] B^T,  A row-major [M][lda], B row-major [N][ldb]
// (B is a weight matrix W [out x in] for the forward, W^T for input gradients),
// with the epilogues of epilogue.cuh.
//
// Register-blocked SGEMM: 128 x BN x 16 block tile (BN = 128 or 64), 256
// threads as 16 x 16, each thread an 8 x (BN / 16) outer-product block (rows
// {4 ty .. 4 ty + 3} and {64 + 4 ty ..}, columns {4 tx ..} and {64 + 4 tx ..}),
// so every shared-memory read is a 16-byte vector and the 16 column groups of a
// warp read 64 consecutive floats.  Operands are read from global memory as
// float4 rows (when the row starts and strides allow it), stored k-major into
// a double-buffered shared-memory tile, and the next k-slice is loaded into
// registers while the current one is multiplied (one barrier per slice).  The
// column tiles of one row block are neighbouring blocks of the grid, so the
// A rows are read from HBM once and the other column tiles hit L2.
#include <cuda_runtime.h>

#include "epilogue.cuh"
#include "internal.h"

namespace alg {

constexpr int SB_M = 128, SB_K = 16, SB_PAD = 4;

// One 4-wide k group of row r (global row index), zero beyond M and K.
__device__ __forceinline__ float4 ld_k4(const float* __restrict__ P, int ld, int rows, int r, int K, int k,
                                        bool vec) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r >= rows) return v;
  const float* p = P + (size_t)r * ld + k;
  if (vec && k + 3 < K) return __ldg(reinterpret_cast<const float4*>(p));
  if (k < K) v.x = __ldg(p);
  if (k + 1 < K) v.y = __ldg(p + 1);
  if (k + 2 < K) v.z = __ldg(p + 2);
  if (k + 3 < K) v.w = __ldg(p + 3);
  return v;
}

// Four consecutive columns [n, n+4) of row m (n + 3 < N, 16-byte aligned rows).
__device__ __forceinline__ void epi_apply4_f32(const EpiParams& ep, int m, int n, float4 a) {
  float v[4] = {a.x, a.y, a.z, a.w};
  if (ep.epi == EPI_FWD_SILU) {
    if (ep.pre) *reinterpret_cast<float4*>(reinterpret_cast<float*>(ep.pre) + (size_t)m * ep.ldp + n) = a;
    const float rs = ep.rowscale ? ep.rowscale[m] : 1.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = v[j] * epi_sigmoid(v[j]) * rs;
  } else if (ep.epi == EPI_F32) {
    if (ep.add) {
      const float4 x = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(ep.add) +
                                                        (size_t)m * ep.ld_add + n);
      v[0] += x.x; v[1] += x.y; v[2] += x.z; v[3] += x.w;
    }
  } else if (ep.epi == EPI_BWD_SILU) {
    const float4 z4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(ep.pre) + (size_t)m * ep.ldp + n);
    const float z[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float s = epi_sigmoid(z[j]);
      v[j] = v[j] * s * (1.0f + z[j] * (1.0f - s));
    }
  }
  *reinterpret_cast<float4*>(reinterpret_cast<float*>(ep.out) + (size_t)m * ep.ldo + n) =
      make_float4(v[0], v[1], v[2], v[3]);
}

template <int BN>
__global__ void __launch_bounds__(256, 2) gemm_simt_kernel(const float* __restrict__ A, int lda,
                                                           const float* __restrict__ B, int ldb, int M, int N,
                                                           int K, EpiParams ep, int vecA, int vecB) {
  constexpr int NJ = BN / 64;                 // column groups of 4 per thread (1 or 2)
  constexpr int BLOADS = BN * SB_K / 4 / 256; // float4 loads of the B slice per thread (1 or 2)
  __shared__ __align__(16) float As[2][SB_K][SB_M + SB_PAD];
  __shared__ __align__(16) float Bs[2][SB_K][BN + SB_PAD];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // linear block index: the column tiles of a row block are consecutive
  const int ntn = (N + BN - 1) / BN;
  const int n0 = (int)(blockIdx.x % ntn) * BN, m0 = (int)(blockIdx.x / ntn) * SB_M;
  // load mapping: row (tid >> 2) (+64), k group (tid & 3) * 4
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  float4 ra[2], rb[BLOADS];
  auto gload = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) ra[h] = ld_k4(A, lda, M, m0 + lr + 64 * h, K, k0 + lk, vecA != 0);
#pragma unroll
    for (int h = 0; h < BLOADS; ++h) rb[h] = ld_k4(B, ldb, N, n0 + lr + 64 * h, K, k0 + lk, vecB != 0);
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      As[buf][lk + 0][lr + 64 * h] = ra[h].x;
      As[buf][lk + 1][lr + 64 * h] = ra[h].y;
      As[buf][lk + 2][lr + 64 * h] = ra[h].z;
      As[buf][lk + 3][lr + 64 * h] = ra[h].w;
    }
#pragma unroll
    for (int h = 0; h < BLOADS; ++h) {
      Bs[buf][lk + 0][lr + 64 * h] = rb[h].x;
      Bs[buf][lk + 1][lr + 64 * h] = rb[h].y;
      Bs[buf][lk + 2][lr + 64 * h] = rb[h].z;
      Bs[buf][lk + 3][lr + 64 * h] = rb[h].w;
    }
  };
  float acc[8][4 * NJ];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4 * NJ; ++j) acc[i][j] = 0.0f;

  const int nk = (K + SB_K - 1) / SB_K;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * SB_K);
#pragma unroll
    for (int k = 0; k < SB_K; ++k) {
      float a[8], b[4 * NJ];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + 4 * ty]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
      for (int jg = 0; jg < NJ; ++jg) {
        const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][k][64 * jg + 4 * tx]);
        b[4 * jg] = bv.x; b[4 * jg + 1] = bv.y; b[4 * jg + 2] = bv.z; b[4 * jg + 3] = bv.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4 * NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + (i - 4));
    if (m >= M) continue;
#pragma unroll
    for (int jg = 0; jg < NJ; ++jg) {
      const int n = n0 + 64 * jg + 4 * tx;
      if (ep.vec && n + 3 < N) {
        epi_apply4_f32(ep, m, n, make_float4(acc[i][4 * jg], acc[i][4 * jg + 1], acc[i][4 * jg + 2],
                                             acc[i][4 * jg + 3]));
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (n + j < N) epi_apply<float>(ep, m, n + j, acc[i][4 * jg + j]);
      }
    }
  }
}

void gemm_simt_f32(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return;
  const float* A = reinterpret_cast<const float*>(g.A);
  const float* B = g.trans ? g.W->f32T : g.W->f32;
  const int ldb = g.trans ? g.W->ldT : g.W->ld;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int vecA = al16(A) && g.lda % 4 == 0;
  const int vecB = al16(B) && ldb % 4 == 0;
  const EpiParams ep = make_epi(g);
  // 128-wide column tiles unless that would leave a half-empty last tile
  const unsigned mt = (unsigned)((g.M + SB_M - 1) / SB_M);
  if (g.N % 128 == 0 || g.N > 512) {
    gemm_simt_kernel<128><<<mt * (unsigned)((g.N + 127) / 128), 256, 0, st>>>(A, g.lda, B, ldb, g.M, g.N, g.K,
                                                                              ep, vecA, vecB);
  } else {
    gemm_simt_kernel<64><<<mt * (unsigned)((g.N + 63) / 64), 256, 0, st>>>(A, g.lda, B, ldb, g.M, g.N, g.K, ep,
                                                                            vecA, vecB);
  }
}

}  // namespace alg
