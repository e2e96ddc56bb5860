// Float32 GEMM on the CUDA cores (the all-float32 path of the MLPs):
//   C[M x N] = A[M x K] B^T,  A row-major [M][lda], B row-major [N][ldb]
// (B is a weight matrix W [out x in] for the forward, W^T for input gradients),
// with the epilogues of epilogue.cuh.  128 x 64 x 16 block tile, 256 threads,
// 8 x 4 outputs per thread, operands staged through shared memory.
#include <cuda_runtime.h>

#include "epilogue.cuh"
#include "internal.h"

namespace alg {

constexpr int SB_M = 128, SB_N = 64, SB_K = 16;

__global__ void __launch_bounds__(256) gemm_simt_kernel(const float* __restrict__ A, int lda,
                                                        const float* __restrict__ B, int ldb, int M, int N,
                                                        int K, EpiParams ep) {
  __shared__ float As[SB_K][SB_M + 4];
  __shared__ float Bs[SB_K][SB_N + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * SB_M, n0 = blockIdx.y * SB_N;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  // load mapping
  const int am = tid >> 1, ak = (tid & 1) * 8;      // A: 128 rows x 16 k, 8 per thread
  const int bn = tid >> 2, bk = (tid & 3) * 4;      // B: 64 rows x 16 k, 4 per thread
  for (int k0 = 0; k0 < K; k0 += SB_K) {
    {
      const int m = m0 + am;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + ak + q;
        As[ak + q][am] = (m < M && k < K) ? A[(size_t)m * lda + k] : 0.0f;
      }
      const int n = n0 + bn;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + bk + q;
        Bs[bk + q][bn] = (n < N && k < K) ? B[(size_t)n * ldb + k] : 0.0f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SB_K; ++k) {
      float a[8], b[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[k][ty * 8 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + ty * 8 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < N) epi_apply<float>(ep, m, n, acc[i][j]);
    }
  }
}

void gemm_simt_f32(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return;
  const float* B = g.trans ? g.W->f32T : g.W->f32;
  const int ldb = g.trans ? g.W->ldT : g.W->ld;
  dim3 grid((g.M + SB_M - 1) / SB_M, (g.N + SB_N - 1) / SB_N);
  gemm_simt_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(g.A), g.lda, B, ldb, g.M, g.N, g.K,
                                         make_epi(g));
}

}  // namespace alg
