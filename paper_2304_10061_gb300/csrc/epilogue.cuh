// GEMM epilogues shared by the float32 SIMT GEMM and the tcgen05 BF16 GEMM.
//   EPI_FWD_SILU  pre[m][n] = acc (if pre);  out[m][n] = silu(acc) * (rowscale ? rowscale[m] : 1)
//   EPI_F32       out[m][n] = acc + (add ? add[m][n] : 0)            (float32 out)
//   EPI_BWD_SILU  out[m][n] = acc * silu'(pre[m][n]),  silu'(z) = s (1 + z (1 - s)), s = sigmoid(z)
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace alg {

struct EpiParams {
  int epi;
  void* out; int ldo;
  void* pre; int ldp;
  const float* rowscale;
  const float* add; int ld_add;
};

__device__ __forceinline__ float act_ld(const float* p) { return *p; }
__device__ __forceinline__ float act_ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void act_st(float* p, float v) { *p = v; }
__device__ __forceinline__ void act_st(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float epi_sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

template <typename T>
__device__ __forceinline__ void epi_apply(const EpiParams& ep, int m, int n, float acc) {
  if (ep.epi == EPI_FWD_SILU) {
    if (ep.pre) act_st(reinterpret_cast<T*>(ep.pre) + (size_t)m * ep.ldp + n, acc);
    float h = acc * epi_sigmoid(acc);
    if (ep.rowscale) h *= ep.rowscale[m];
    act_st(reinterpret_cast<T*>(ep.out) + (size_t)m * ep.ldo + n, h);
  } else if (ep.epi == EPI_F32) {
    float v = acc;
    if (ep.add) v += ep.add[(size_t)m * ep.ld_add + n];
    reinterpret_cast<float*>(ep.out)[(size_t)m * ep.ldo + n] = v;
  } else {
    float z = act_ld(reinterpret_cast<const T*>(ep.pre) + (size_t)m * ep.ldp + n);
    float s = epi_sigmoid(z);
    act_st(reinterpret_cast<T*>(ep.out) + (size_t)m * ep.ldo + n, acc * s * (1.0f + z * (1.0f - s)));
  }
}

inline EpiParams make_epi(const GemmArgs& g) {
  EpiParams e;
  e.epi = g.epi; e.out = g.out; e.ldo = g.ldo; e.pre = g.pre; e.ldp = g.ldp;
  e.rowscale = g.rowscale; e.add = g.add; e.ld_add = g.ld_add;
  return e;
}

}  // namespace alg
