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
  const void* add; int ld_add;   // float (EPI_F32), bf16 (EPI_HEAD, tcgen05 path)
  int vec;   // 1: every row start of out/pre/add is 16-byte aligned (vector path allowed)
  float* ubar;
  const float* v;
  const float* rowsig;
  float* Eout;
};

__device__ __forceinline__ float act_ld(const float* p) { return *p; }
__device__ __forceinline__ float act_ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void act_st(float* p, float v) { *p = v; }
__device__ __forceinline__ void act_st(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float epi_sigmoid(float z) { return __fdividef(1.0f, 1.0f + expf(-z)); }

template <typename T>
__device__ __forceinline__ void epi_apply(const EpiParams& ep, int m, int n, float acc) {
  if (ep.epi == EPI_FWD_SILU) {
    if (ep.pre) act_st(reinterpret_cast<T*>(ep.pre) + (size_t)m * ep.ldp + n, acc);
    float h = acc * epi_sigmoid(acc);
    if (ep.rowscale) h *= ep.rowscale[m];
    act_st(reinterpret_cast<T*>(ep.out) + (size_t)m * ep.ldo + n, h);
  } else if (ep.epi == EPI_F32) {
    float v = acc;
    if (ep.add) v += reinterpret_cast<const float*>(ep.add)[(size_t)m * ep.ld_add + n];
    reinterpret_cast<float*>(ep.out)[(size_t)m * ep.ldo + n] = v;
  } else if (ep.epi == EPI_LINEAR) {
    act_st(reinterpret_cast<T*>(ep.out) + (size_t)m * ep.ldo + n, acc);
  } else {
    float z = act_ld(reinterpret_cast<const T*>(ep.pre) + (size_t)m * ep.ldp + n);
    float s = epi_sigmoid(z);
    act_st(reinterpret_cast<T*>(ep.out) + (size_t)m * ep.ldo + n, acc * s * (1.0f + z * (1.0f - s)));
  }
}

// 32 consecutive columns [n, n+32) of row m, bf16 activations, 16-byte vector I/O.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void store_bf16x32(bf16* p, const float (&v)[32]) {
  uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    q[k] = make_uint4(pack_bf16x2(v[8 * k + 0], v[8 * k + 1]), pack_bf16x2(v[8 * k + 2], v[8 * k + 3]),
                      pack_bf16x2(v[8 * k + 4], v[8 * k + 5]), pack_bf16x2(v[8 * k + 6], v[8 * k + 7]));
}

__device__ __forceinline__ void load_bf16x32(const bf16* p, float (&v)[32]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint4 x = q[k];
    uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w[t]);
      float2 f = __bfloat1622float2(h);
      v[8 * k + 2 * t] = f.x;
      v[8 * k + 2 * t + 1] = f.y;
    }
  }
}

__device__ __forceinline__ void epi_apply_vec32_bf16(const EpiParams& ep, int m, int n, float (&v)[32]) {
  if (ep.epi == EPI_FWD_SILU) {
    if (ep.pre) store_bf16x32(reinterpret_cast<bf16*>(ep.pre) + (size_t)m * ep.ldp + n, v);
    const float rs = ep.rowscale ? ep.rowscale[m] : 1.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = v[j] * epi_sigmoid(v[j]) * rs;
    store_bf16x32(reinterpret_cast<bf16*>(ep.out) + (size_t)m * ep.ldo + n, v);
  } else if (ep.epi == EPI_F32) {
    float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(ep.out) + (size_t)m * ep.ldo + n);
    if (ep.add) {
      const float4* a = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(ep.add) + (size_t)m * ep.ld_add + n);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float4 x = a[k];
        o[k] = make_float4(v[4 * k] + x.x, v[4 * k + 1] + x.y, v[4 * k + 2] + x.z, v[4 * k + 3] + x.w);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
  } else {
    float z[32];
    load_bf16x32(reinterpret_cast<const bf16*>(ep.pre) + (size_t)m * ep.ldp + n, z);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float s = epi_sigmoid(z[j]);
      v[j] = v[j] * s * (1.0f + z[j] * (1.0f - s));
    }
    store_bf16x32(reinterpret_cast<bf16*>(ep.out) + (size_t)m * ep.ldo + n, v);
  }
}

inline EpiParams make_epi(const GemmArgs& g) {
  EpiParams e;
  e.epi = g.epi; e.out = g.out; e.ldo = g.ldo; e.pre = g.pre; e.ldp = g.ldp;
  e.rowscale = g.rowscale; e.add = g.add; e.ld_add = g.ld_add;
  e.ubar = g.ubar; e.v = g.v; e.rowsig = g.rowsig; e.Eout = g.Eout;
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  e.vec = al(g.out) && al(g.pre) && al(g.add) && (g.ldo % 8 == 0) && (g.ldp % 8 == 0) && (g.ld_add % 8 == 0);
  return e;
}

}  // namespace alg
