// Per-edge and per-atom kernels that are not GEMMs or environment sums:
//   edge geometry and basis (forward and adjoint), the elementwise head of each
//   MLP's adjoint, the edge energy, and the float64 atom/structure reductions.
//
// Basis (Sec. "Training details": 8 Bessel functions and a polynomial envelope,
// details as in the Allegro paper; readings fixed by this library):
//   B_n(r) = sqrt(2/r_c) sin(n pi r / r_c) / r,  n = 1..n_bessel
//   u(x)   = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2),  x = r / r_c
// Real spherical harmonics, component-normalised (sum_m Y_lm^2 = 2l+1), of the
// unit vector (x, y, z) = r_hat:
//   l=0: 1
//   l=1: sqrt3 y, sqrt3 z, sqrt3 x
//   l=2: sqrt15 xy, sqrt15 yz, sqrt5/2 (3z^2 - 1), sqrt15 xz, sqrt15/2 (x^2 - y^2)
//   l=3: c3 y (3x^2 - y^2), 2 c2 xyz, c1 (15z^2 - 3) y, c0 z (5z^2 - 3), c1 (15z^2 - 3) x,
//        c2 z (x^2 - y^2), c3 x (x^2 - 3y^2);  c0 = sqrt7/2, c1 = sqrt(7/6)/2,
//        c2 = 15 sqrt(7/60), c3 = 15 sqrt(7/360)
// Two-body input row: [onehot(Z_i) | onehot(Z_j) | B(r)].
#include <cuda_runtime.h>

#include <algorithm>
#include <cuda_bf16.h>

#include "amax.cuh"
#include "internal.h"

namespace alg {

template <typename T> __device__ __forceinline__ T to_act(float v);
template <> __device__ __forceinline__ float to_act<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 to_act<bf16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from_act(float v) { return v; }
__device__ __forceinline__ float from_act(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(bf16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float sigmoidf_(float z) { return __fdividef(1.0f, 1.0f + expf(-z)); }

struct BasisConst {
  int ns, nb, p, lmax, S;
  float rc, inv_rc, pref;       // pref = sqrt(2/r_c)
  float c0, c1, c2;             // envelope coefficients
  const float2* pair;           // per ordered species pair {1/rc, sqrt(2/rc)}, or null (rc for every pair)
};

// 1/rc and sqrt(2/rc) of the ordered pair (Z_i, Z_j)
__device__ __forceinline__ float2 pair_basis(const BasisConst& bc, int zi, int zj) {
  return bc.pair ? bc.pair[zi * bc.ns + zj] : make_float2(bc.inv_rc, bc.pref);
}

static BasisConst make_basis(const Arch& a) {
  BasisConst b;
  b.ns = a.ns; b.nb = a.nb; b.p = a.p; b.lmax = a.lmax; b.S = a.S();
  b.rc = (float)a.rc; b.inv_rc = (float)(1.0 / a.rc); b.pref = (float)sqrt(2.0 / a.rc);
  b.c0 = (float)((a.p + 1.0) * (a.p + 2.0) / 2.0);
  b.c1 = (float)(a.p * (a.p + 2.0));
  b.c2 = (float)(a.p * (a.p + 1.0) / 2.0);
  b.pair = reinterpret_cast<const float2*>(a.pair_basis);
  return b;
}

__device__ __forceinline__ float ipow(float x, int p) {
  float r = 1.0f;
  for (int k = 0; k < p; ++k) r *= x;
  return r;
}

__device__ __forceinline__ void sh_eval(int lmax, float x, float y, float z, float* Y) {
  const float s3 = 1.7320508075688772f, s15 = 3.8729833462074170f, s5h = 1.1180339887498949f;
  Y[0] = 1.0f;
  if (lmax >= 1) { Y[1] = s3 * y; Y[2] = s3 * z; Y[3] = s3 * x; }
  if (lmax >= 2) {
    Y[4] = s15 * x * y; Y[5] = s15 * y * z; Y[6] = s5h * (3.0f * z * z - 1.0f);
    Y[7] = s15 * x * z; Y[8] = 0.5f * s15 * (x * x - y * y);
  }
  if (lmax >= 3) {
    // N_l|m| d^|m|P_3/dz^|m| A_m with the normalisation sqrt(7 (2 - d_m0) (3-|m|)! / (3+|m|)!)
    const float c0 = 1.3228756555322954f;   // sqrt(7) / 2
    const float c1 = 0.5400617248673217f;   // sqrt(7/6) / 2
    const float c2 = 5.1234753829797990f;   // 15 sqrt(7/60)
    const float c3 = 2.0916500663351889f;   // 15 sqrt(7/360)
    const float f = 15.0f * z * z - 3.0f;
    Y[9] = c3 * y * (3.0f * x * x - y * y);
    Y[10] = 2.0f * c2 * x * y * z;
    Y[11] = c1 * f * y;
    Y[12] = c0 * z * (5.0f * z * z - 3.0f);
    Y[13] = c1 * f * x;
    Y[14] = c2 * z * (x * x - y * y);
    Y[15] = c3 * x * (x * x - 3.0f * y * y);
  }
}

// sum_a Ybar_a grad Y_a (gradient of the polynomial forms above w.r.t. (x, y, z))
__device__ __forceinline__ void sh_vjp(int lmax, float x, float y, float z, const float* Yb, float G[3]) {
  const float s3 = 1.7320508075688772f, s15 = 3.8729833462074170f, s5 = 2.2360679774997897f;
  G[0] = G[1] = G[2] = 0.0f;
  if (lmax >= 1) { G[1] += s3 * Yb[1]; G[2] += s3 * Yb[2]; G[0] += s3 * Yb[3]; }
  if (lmax >= 2) {
    G[0] += s15 * (Yb[4] * y + Yb[7] * z + Yb[8] * x);
    G[1] += s15 * (Yb[4] * x + Yb[5] * z - Yb[8] * y);
    G[2] += s15 * (Yb[5] * y + Yb[7] * x) + 3.0f * s5 * Yb[6] * z;
  }
  if (lmax >= 3) {
    const float c0 = 1.3228756555322954f, c1 = 0.5400617248673217f, c2 = 5.1234753829797990f,
                c3 = 2.0916500663351889f;
    const float f = 15.0f * z * z - 3.0f;
    G[0] += c3 * Yb[9] * 6.0f * x * y + 2.0f * c2 * Yb[10] * y * z + c1 * Yb[13] * f +
            c2 * Yb[14] * 2.0f * x * z + c3 * Yb[15] * 3.0f * (x * x - y * y);
    G[1] += c3 * Yb[9] * 3.0f * (x * x - y * y) + 2.0f * c2 * Yb[10] * x * z + c1 * Yb[11] * f -
            c2 * Yb[14] * 2.0f * y * z - c3 * Yb[15] * 6.0f * x * y;
    G[2] += 2.0f * c2 * Yb[10] * x * y + c1 * Yb[11] * 30.0f * z * y + c0 * Yb[12] * f +
            c1 * Yb[13] * 30.0f * z * x + c2 * Yb[14] * (x * x - y * y);
  }
}

// Sigmoid of the path's MLP epilogues: the BF16 path's GEMMs use the hardware
// tanh approximation, sigma(z) = (1 + tanh(z/2)) / 2, the float32 path the
// exponential form; the fused first layer uses the same one as its adjoint.
template <typename T> __device__ __forceinline__ float path_sigmoid(float z);
template <> __device__ __forceinline__ float path_sigmoid<float>(float z) { return sigmoidf_(z); }
template <> __device__ __forceinline__ float path_sigmoid<bf16>(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return fmaf(0.5f, t, 0.5f);
}

// Edge geometry, basis and the first two-body layer, one block of kGeomBlock
// edges.  The layer's input row [onehot(Z_i) | onehot(Z_j) | B(r)] is never
// formed: z_k = W0[k][Z_i] + W0[k][ns + Z_j] + sum_n W0[k][2 ns + n] B_n(r),
// with W0 read as its transpose W0t[input][output] from shared memory, 32
// output columns at a time.  Outputs: Y, u, sigma_{Z_i}, the pre-activation
// z and the activation silu(z) (times u when the layer is the MLP's last), all
// staged in shared memory and written back as contiguous runs (per-thread
// records would scatter over partial sectors).
constexpr int kGeomBlock = 128;
constexpr int kGeomCols = 32;                   // output columns per pass
constexpr int kGeomWPad = kGeomCols + 4;        // padded shared row of W0t (float4-aligned, bank-spread)

template <typename T>
__host__ __device__ constexpr int geom_stage_ld() { return kGeomCols + 16 / (int)sizeof(T); }   // padded row, 16-byte multiple

// four consecutive activation-type values from floats (8- or 16-byte aligned)
__device__ __forceinline__ void st4_act(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4_act(bf16* p, const float (&v)[4]) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
}

template <typename T>
__device__ __forceinline__ void copy_rows_out(const T* src, int lds, T* dst, int ldd, int c0, int nrows, int nc) {
  // rows of nc elements from shared (row pitch lds) to global (row pitch ldd, column offset c0)
  const bool vec = ((nc * (int)sizeof(T)) % 16 == 0) && ((c0 * (int)sizeof(T)) % 16 == 0) &&
                   ((ldd * (int)sizeof(T)) % 16 == 0);
  if (vec) {
    const int per = nc * (int)sizeof(T) / 16;
    for (int q = threadIdx.x; q < nrows * per; q += blockDim.x) {
      const int rr = q / per, cc = q - rr * per;
      reinterpret_cast<uint4*>(dst + (size_t)rr * ldd + c0)[cc] = reinterpret_cast<const uint4*>(src + rr * lds)[cc];
    }
  } else {
    for (int q = threadIdx.x; q < nrows * nc; q += blockDim.x) {
      const int rr = q / nc, cc = q - rr * nc;
      dst[(size_t)rr * ldd + c0 + cc] = src[rr * lds + cc];
    }
  }
}

// AMAX: record max|activation| for the FP8 per-tensor scale (the other paths skip the work)
template <typename T, bool AMAX>
__global__ void __launch_bounds__(kGeomBlock)
    geom_fwd_kernel(int Ec, int e0, const double* __restrict__ ed, const int* __restrict__ ei,
                    const int* __restrict__ ej, const int* __restrict__ species, BasisConst bc,
                    float* __restrict__ Yout, float* __restrict__ uout, const double* __restrict__ sigma,
                    float* __restrict__ sig, const float* __restrict__ W0t, int ldW, int N0, T* __restrict__ Zout,
                    int ldZ, T* __restrict__ Hout, int ldH, int scale_u, unsigned* __restrict__ amax) {
  constexpr int LDS = geom_stage_ld<T>();
  extern __shared__ __align__(16) uint8_t geom_sm[];
  const int K0 = 2 * bc.ns + bc.nb;
  const int WP = kGeomWPad;   // shared row pitch of W0t (floats)
  float* sY = reinterpret_cast<float*>(geom_sm);                                  // [kGeomBlock][kMaxS]
  float* sW = sY + kGeomBlock * kMaxS;                                            // [K0][WP]
  T* sZ = reinterpret_cast<T*>(sW + K0 * WP);                                     // [kGeomBlock][LDS]
  T* sH = sZ + kGeomBlock * LDS;                                                  // [kGeomBlock][LDS]
  const int tl = threadIdx.x;
  const int ntiles = (Ec + kGeomBlock - 1) / kGeomBlock;
  float hmax = 0.0f;   // max |activation| written (FP8 per-tensor scale)
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int eb = tile * kGeomBlock;
    const int nloc = min(kGeomBlock, Ec - eb);
    const int e = eb + tl;
    float B[kMaxBessel];
    float u = 0.0f;
    int zi = 0, zj = 0;
    __syncthreads();   // the previous tile's Y staging has been copied out
    if (tl < nloc) {
      const size_t eg = (size_t)e0 + e;
      const double dx = ed[3 * eg], dy = ed[3 * eg + 1], dz = ed[3 * eg + 2];
      // float32 geometry from the exact float64 displacement
      const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
      const float r2 = fx * fx + fy * fy + fz * fz;
      const float ir32 = rsqrtf(r2);
      const float r = r2 * ir32;
      const float x = fx * ir32, y = fy * ir32, z = fz * ir32;
      float Y[kMaxS];
      sh_eval(bc.lmax, x, y, z, Y);
#pragma unroll
      for (int a = 0; a < kMaxS; ++a)
        if (a < bc.S) sY[tl * bc.S + a] = Y[a];
      zi = species[ei[eg]];
      zj = species[ej[eg]];
      const float2 pb = pair_basis(bc, zi, zj);   // the pair's 1/rc and sqrt(2/rc)
      const float xr = r * pb.x;
      if (xr < 1.0f) {
        const float xp = ipow(xr, bc.p);
        u = 1.0f - xp * (bc.c0 - xr * (bc.c1 - bc.c2 * xr));
      }
      uout[e] = u;
      if (sig) sig[e] = (float)sigma[zi];
      // sin(n pi x) for n = 1..nb by the angle-addition recurrence from one
      // sincospi: (s, c)_{n+1} = (s_n c_1 + c_n s_1, c_n c_1 - s_n s_1)
      float s1, c1;
      sincospif(xr, &s1, &c1);
      float sn = s1, cn = c1;
#pragma unroll
      for (int n = 0; n < kMaxBessel; ++n) {
        B[n] = (n < bc.nb) ? pb.y * sn * ir32 : 0.0f;
        const float s2 = fmaf(sn, c1, cn * s1);
        cn = fmaf(cn, c1, -(sn * s1));
        sn = s2;
      }
    }
    const float rsc = scale_u ? u : 1.0f;
    for (int c0 = 0; c0 < N0; c0 += kGeomCols) {
      const int nc = min(kGeomCols, N0 - c0);
      __syncthreads();   // the previous pass's staging has been copied out
      for (int q = tl; q < K0 * kGeomCols; q += kGeomBlock) {
        const int rr = q / kGeomCols, cc = q - rr * kGeomCols;
        sW[rr * kGeomWPad + cc] = (cc < nc) ? W0t[(size_t)rr * ldW + c0 + cc] : 0.0f;
      }
      __syncthreads();
      if (tl < nloc) {
        const float* wi = sW + zi * WP;
        const float* wj = sW + (bc.ns + zj) * WP;
        const float* wb = sW + 2 * bc.ns * WP;
#pragma unroll 2
        for (int c4 = 0; c4 < kGeomCols; c4 += 4) {
          const float4 a = *reinterpret_cast<const float4*>(wi + c4);
          const float4 b = *reinterpret_cast<const float4*>(wj + c4);
          // column pairs in packed fp32 (FFMA2 / FMUL2: each half the ordinary
          // IEEE fp32 fma / multiply, so the results equal the scalar ones)
          float2 z01 = make_float2(a.x + b.x, a.y + b.y), z23 = make_float2(a.z + b.z, a.w + b.w);
#pragma unroll
          for (int n = 0; n < kMaxBessel; ++n) {
            if (n < bc.nb) {
              const float4 w = *reinterpret_cast<const float4*>(wb + n * WP + c4);
              const float2 bn = make_float2(B[n], B[n]);
              z01 = __ffma2_rn(bn, make_float2(w.x, w.y), z01);
              z23 = __ffma2_rn(bn, make_float2(w.z, w.w), z23);
            }
          }
          const float2 rs2 = make_float2(rsc, rsc);
          const float2 g01 = make_float2(path_sigmoid<T>(z01.x), path_sigmoid<T>(z01.y));
          const float2 g23 = make_float2(path_sigmoid<T>(z23.x), path_sigmoid<T>(z23.y));
          const float2 h01 = __fmul2_rn(__fmul2_rn(z01, g01), rs2);
          const float2 h23 = __fmul2_rn(__fmul2_rn(z23, g23), rs2);
          const float acc[4] = {z01.x, z01.y, z23.x, z23.y};
          const float hv[4] = {h01.x, h01.y, h23.x, h23.y};
          if constexpr (AMAX) {
#pragma unroll
            for (int k = 0; k < 4; ++k) hmax = fmaxf(hmax, fabsf(hv[k]));
          }
          st4_act(sZ + tl * LDS + c4, acc);
          st4_act(sH + tl * LDS + c4, hv);
        }
      }
      __syncthreads();
      copy_rows_out<T>(sZ, LDS, Zout + (size_t)eb * ldZ, ldZ, c0, nloc, nc);
      copy_rows_out<T>(sH, LDS, Hout + (size_t)eb * ldH, ldH, c0, nloc, nc);
    }
    // Y: nloc * S floats starting at float eb * S (4-byte aligned only): scalar, coalesced
    float* dst = Yout + (size_t)eb * bc.S;
    for (int q = tl; q < nloc * bc.S; q += kGeomBlock) dst[q] = sY[q];
  }
  if constexpr (AMAX) record_amax(amax, hmax);
}

template <typename T>
void edge_geom_fwd(int Ec, int e0, const double* ed, const int* ei, const int* ej, const int* species,
                   const Arch& a, float* Y, float* u, const double* sigma, float* sig, const float* W0t, int ldW,
                   T* Z0, int ldZ, T* H0, int ldH, bool scale_u, cudaStream_t st, unsigned* amax) {
  if (Ec <= 0) return;
  const int N0 = a.tb[0], K0 = a.K0in();
  const size_t stage = (size_t)kGeomBlock * kMaxS * 4 + 2 * (size_t)kGeomBlock * geom_stage_ld<T>() * sizeof(T);
  const int tiles = (Ec + kGeomBlock - 1) / kGeomBlock;
  // one tile per block, 32 weight columns staged per pass (measured faster than persistent
  // blocks holding all of W0t)
  const size_t smem = stage + (size_t)K0 * kGeomWPad * 4;
  auto launch = [&](auto kern) {
    if (smem > 48 * 1024)   // many species: opt in to more than the default dynamic shared memory
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<tiles, kGeomBlock, smem, st>>>(Ec, e0, ed, ei, ej, species, make_basis(a), Y, u, sigma, sig, W0t, ldW, N0,
                                          Z0, ldZ, H0, ldH, scale_u ? 1 : 0, amax);
  };
  if (amax) launch(geom_fwd_kernel<T, true>);
  else launch(geom_fwd_kernel<T, false>);
}
template void edge_geom_fwd<float>(int, int, const double*, const int*, const int*, const int*, const Arch&,
                                   float*, float*, const double*, float*, const float*, int, float*, int, float*,
                                   int, bool, cudaStream_t, unsigned*);
template void edge_geom_fwd<bf16>(int, int, const double*, const int*, const int*, const int*, const Arch&,
                                  float*, float*, const double*, float*, const float*, int, bf16*, int, bf16*, int,
                                  bool, cudaStream_t, unsigned*);

// Adjoint of the geometry.  The first two-body layer's input adjoint is only
// needed for its Bessel part: Bbar_n = sum_k zbar0_k W0[k][2 ns + n] (the
// one-hot species inputs carry no geometry), formed here from zbar0 and the
// Bessel rows of W0t held in shared memory.
constexpr int kGeomBwdBlocksPerSM = 8;
template <typename T>
__global__ void __launch_bounds__(kGeomBlock, kGeomBwdBlocksPerSM)
    geom_bwd_kernel(int Ec, int e0, const double* __restrict__ ed, const int* __restrict__ ei,
                    const int* __restrict__ ej, const int* __restrict__ species, BasisConst bc,
                    const T* __restrict__ zbar0,
                    int ldz, const float* __restrict__ W0t, int ldW, int N0, const float* __restrict__ ubar,
                    YbarParts yb, float* __restrict__ g) {
  extern __shared__ __align__(16) float wb_sm[];   // [nb][N0]: Bessel rows of W0t
  for (int q = threadIdx.x; q < bc.nb * N0; q += blockDim.x) {
    const int n = q / N0, k = q - n * N0;
    wb_sm[q] = W0t[(size_t)(2 * bc.ns + n) * ldW + k];
  }
  __syncthreads();
  // persistent blocks (a few per SM): the Bessel rows are staged once per block
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ec; e += gridDim.x * blockDim.x) {
    const size_t eg = (size_t)e0 + e;
    const double dx = ed[3 * eg], dy = ed[3 * eg + 1], dz = ed[3 * eg + 2];
    // float32 geometry from the exact float64 displacement
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    const float r2 = fx * fx + fy * fy + fz * fz;
    const float ir32 = rsqrtf(r2);
    const float r = r2 * ir32;
    const float x = fx * ir32, y = fy * ir32, z = fz * ir32;
    const float2 pb = pair_basis(bc, bc.pair ? species[ei[eg]] : 0, bc.pair ? species[ej[eg]] : 0);
    const float inv_rc = pb.x, pref = pb.y;
    const float xr = r * inv_rc;
    // Bbar = zbar0 . W0[:, 2 ns:]
    float Bb[kMaxBessel];
  #pragma unroll
    for (int n = 0; n < kMaxBessel; ++n) Bb[n] = 0.0f;
    const T* zr = zbar0 + (size_t)e * ldz;
    constexpr int V = 16 / (int)sizeof(T);   // elements per 16-byte vector
    int k0 = 0;
    if ((ldz * (int)sizeof(T)) % 16 == 0 && N0 % 4 == 0) {   // 16-byte aligned rows: vector loads
      for (; k0 + V <= N0; k0 += V) {
        const uint4 q = *reinterpret_cast<const uint4*>(zr + k0);
        const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
        float zk[V];
        if constexpr (sizeof(T) == 2) {
  #pragma unroll
          for (int t = 0; t < 4; ++t) {
            zk[2 * t] = __uint_as_float(wv[t] << 16);
            zk[2 * t + 1] = __uint_as_float(wv[t] & 0xffff0000u);
          }
        } else {
  #pragma unroll
          for (int t = 0; t < 4; ++t) zk[t] = __uint_as_float(wv[t]);
        }
  #pragma unroll
        for (int n = 0; n < kMaxBessel; ++n) {
          if (n < bc.nb) {
  #pragma unroll
            for (int v4 = 0; v4 < V; v4 += 4) {   // weight rows are float4-aligned (N0 % 4 == 0 on this path)
              const float4 wv4 = *reinterpret_cast<const float4*>(wb_sm + n * N0 + k0 + v4);
              Bb[n] += zk[v4] * wv4.x + zk[v4 + 1] * wv4.y + zk[v4 + 2] * wv4.z + zk[v4 + 3] * wv4.w;
            }
          }
        }
      }
    }
    for (int k = k0; k < N0; ++k) {
      const float zk = to_f32(zr[k]);
  #pragma unroll
      for (int n = 0; n < kMaxBessel; ++n)
        if (n < bc.nb) Bb[n] += zk * wb_sm[n * N0 + k];
    }
    // dE/dr from the Bessel basis and the envelope
    float dEdr = 0.0f;
    {
      // sin, cos(n pi x) for n = 1..nb by the angle-addition recurrence from one sincospi
      float s1, c1;
      sincospif(xr, &s1, &c1);
      float sn = s1, cn = c1;
  #pragma unroll
      for (int n = 1; n <= kMaxBessel; ++n) {
        if (n > bc.nb) break;
        const float kk = (float)n * 3.14159265358979323846f * inv_rc;
        const float dB = pref * (kk * cn * r - sn) * ir32 * ir32;
        dEdr += Bb[n - 1] * dB;
        const float s2 = fmaf(sn, c1, cn * s1);
        cn = fmaf(cn, c1, -(sn * s1));
        sn = s2;
      }
    }
    if (xr < 1.0f) {
      const float xp1 = ipow(xr, bc.p - 1);
      const float du = xp1 * (-(float)bc.p * bc.c0 + xr * ((float)(bc.p + 1) * bc.c1 - (float)(bc.p + 2) * bc.c2 * xr));
      dEdr += ubar[e] * du * inv_rc;
    }
    // Ybar arrives in two partial arrays (from two row-kernel passes), summed in a fixed order
    float Yb[kMaxS];
  #pragma unroll
    for (int a = 0; a < kMaxS; ++a)
      Yb[a] = (a < bc.S) ? yb.p[0][(size_t)e * bc.S + a] + (yb.p[1] ? yb.p[1][(size_t)e * bc.S + a] : 0.0f) : 0.0f;
    float G[3];
    sh_vjp(bc.lmax, x, y, z, Yb, G);
    const float rg = x * G[0] + y * G[1] + z * G[2];
    g[3 * eg] = x * dEdr + (G[0] - x * rg) * ir32;
    g[3 * eg + 1] = y * dEdr + (G[1] - y * rg) * ir32;
    g[3 * eg + 2] = z * dEdr + (G[2] - z * rg) * ir32;
  }
}

template <typename T>
void edge_geom_bwd(int Ec, int e0, const double* ed, const int* ei, const int* ej, const int* species,
                   const Arch& a, const T* zbar0, int ldz, const float* W0t, int ldW, const float* ubar,
                   const YbarParts& yb, float* g, cudaStream_t st) {
  if (Ec <= 0) return;
  const size_t smem = (size_t)a.nb * a.tb[0] * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(geom_bwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (Ec + kGeomBlock - 1) / kGeomBlock;
  const int grid = std::min(tiles, std::max(nsm, 1) * kGeomBwdBlocksPerSM);
  geom_bwd_kernel<T><<<grid, kGeomBlock, smem, st>>>(
      Ec, e0, ed, ei, ej, species, make_basis(a), zbar0, ldz, W0t, ldW, a.tb[0], ubar, yb, g);
}
template void edge_geom_bwd<float>(int, int, const double*, const int*, const int*, const int*, const Arch&,
                                   const float*, int, const float*, int, const float*, const YbarParts&, float*,
                                   cudaStream_t);
template void edge_geom_bwd<bf16>(int, int, const double*, const int*, const int*, const int*, const Arch&,
                                  const bf16*, int, const float*, int, const float*, const YbarParts&, float*,
                                  cudaStream_t);

// Adjoint head of an MLP whose output is x = u * silu(z):  given xbar,
//   ubar += sum_n xbar_n silu(z_n),   zbar_n = xbar_n u silu'(z_n).
// xbar = sigma_{Z_i} v when `xbar` is null (the last layer: E_ij = v . x with
// the linear edge-energy MLP folded into v, and dE/dE_ij = sigma_{Z_i}).
// four consecutive activation-type values as floats (16-byte float / 8-byte bf16 access)
__device__ __forceinline__ float4 ld4_act(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4_act(const bf16* p) {
  const uint2 w = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4_act4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4_act4(bf16* p, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 w;
  w.x = *reinterpret_cast<const unsigned*>(&a);
  w.y = *reinterpret_cast<const unsigned*>(&b);
  *reinterpret_cast<uint2*>(p) = w;
}

// Adjoint head of an MLP whose output is x = u * silu(z):  given xbar,
//   ubar += sum_n xbar_n silu(z_n),   zbar_n = xbar_n u silu'(z_n).
// xbar = sigma_{Z_i} v when `xbar` is null (the last layer: E_ij = v . x with
// the linear edge-energy MLP folded into v, and dE/dE_ij = sigma_{Z_i}).
// One warp per edge; with `vec` (every row start 16-byte aligned for float,
// 8-byte for bf16) a lane takes four consecutive columns per step.
template <typename T>
__global__ void head_bwd_kernel(int Ec, int K, const float* __restrict__ xbar, int ld_x,
                                const float* __restrict__ vconst, const int* __restrict__ ei,
                                const int* __restrict__ species, const double* __restrict__ sigma, int e0,
                                const T* __restrict__ pre, int ld_pre,
                                const float* __restrict__ u, float* __restrict__ ubar, bool ubar_init,
                                T* __restrict__ zbar, int ld_z, unsigned* __restrict__ amax,
                                const T* __restrict__ addx, int ld_addx, int vec) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= Ec) return;
  const int e = warp;
  float sc = 1.0f;
  if (!xbar) sc = (float)sigma[species[ei[(size_t)e0 + e]]];
  const float ue = u[e];
  float dot = 0.0f, zmax = 0.0f;
  auto one = [&](float xb, float z) -> float {
    const float s = sigmoidf_(z);
    dot += xb * z * s;
    const float zb = xb * ue * s * (1.0f + z * (1.0f - s));
    zmax = fmaxf(zmax, fabsf(zb));
    return zb;
  };
  int n0 = 0;
  if (vec) {
    const int K4 = K & ~3;
#pragma unroll 4
    for (int n = 4 * lane; n < K4; n += 128) {
      float4 xb = xbar ? ld4_act(xbar + (size_t)e * ld_x + n) : ld4_act(vconst + n);
      if (!xbar) { xb.x *= sc; xb.y *= sc; xb.z *= sc; xb.w *= sc; }
      if (addx) {
        const float4 a = ld4_act(addx + (size_t)e * ld_addx + n);
        xb.x += a.x; xb.y += a.y; xb.z += a.z; xb.w += a.w;
      }
      const float4 z = ld4_act(pre + (size_t)e * ld_pre + n);
      float4 zb;
      zb.x = one(xb.x, z.x);
      zb.y = one(xb.y, z.y);
      zb.z = one(xb.z, z.z);
      zb.w = one(xb.w, z.w);
      st4_act4(zbar + (size_t)e * ld_z + n, zb);
    }
    n0 = K4;
  }
  for (int n = n0 + lane; n < K; n += 32) {
    float xb = xbar ? xbar[(size_t)e * ld_x + n] : sc * vconst[n];
    if (addx) xb += from_act(addx[(size_t)e * ld_addx + n]);
    zbar[(size_t)e * ld_z + n] = to_act<T>(one(xb, from_act(pre[(size_t)e * ld_pre + n])));
  }
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) ubar[e] = ubar_init ? dot : ubar[e] + dot;
  record_amax(amax, zmax);
}

template <typename T>
void mlp_head_bwd(int Ec, int K, const float* xbar, int ld_x, const float* vconst, const int* ei,
                  const int* species, const double* sigma, int e0, const T* pre, int ld_pre, const float* u,
                  float* ubar, bool ubar_init, T* zbar, int ld_z, cudaStream_t st, unsigned* amax, const T* addx,
                  int ld_addx) {
  if (Ec <= 0) return;
  long long threads = (long long)Ec * 32;
  auto al = [](const void* p, int b) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) % b) == 0; };
  constexpr int b4 = 4 * (int)sizeof(T);   // bytes of four activation-type values
  const int vec = al(xbar, 16) && al(vconst, 16) && al(pre, b4) && al(zbar, b4) && al(addx, b4) &&
                  (ld_x % 4 == 0) && (ld_pre % 4 == 0) && (ld_z % 4 == 0) && (!addx || ld_addx % 4 == 0);
  head_bwd_kernel<T><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      Ec, K, xbar, ld_x, vconst, ei, species, sigma, e0, pre, ld_pre, u, ubar, ubar_init, zbar, ld_z, amax, addx,
      ld_addx, vec);
}
template void mlp_head_bwd<float>(int, int, const float*, int, const float*, const int*, const int*,
                                  const double*, int, const float*, int, const float*, float*, bool, float*, int,
                                  cudaStream_t, unsigned*, const float*, int);
template void mlp_head_bwd<bf16>(int, int, const float*, int, const float*, const int*, const int*,
                                 const double*, int, const bf16*, int, const float*, float*, bool, bf16*, int,
                                 cudaStream_t, unsigned*, const bf16*, int);

// E_ij = v . x (the linear edge-energy MLP folded into one vector v)
template <typename T>
__global__ void edge_energy_kernel(int Ec, int K, const T* __restrict__ x, int ldx, const float* __restrict__ v,
                                   float* __restrict__ Ee) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= Ec) return;
  float s = 0.0f;
  for (int n = lane; n < K; n += 32) s += from_act(x[(size_t)warp * ldx + n]) * v[n];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Ee[warp] = s;
}

template <typename T>
void edge_energy(int Ec, int K, const T* x, int ldx, const float* v, float* Ee, cudaStream_t st) {
  if (Ec <= 0) return;
  long long threads = (long long)Ec * 32;
  edge_energy_kernel<T><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(Ec, K, x, ldx, v, Ee);
}
template void edge_energy<float>(int, int, const float*, int, const float*, float*, cudaStream_t);
template void edge_energy<bf16>(int, int, const bf16*, int, const float*, float*, cudaStream_t);

// ZBL repulsion of one ordered edge (Sec. "Training details": a Ziegler-
// Biersack-Littmark term is added to the potential).  The universal ZBL pair
// energy k_e Z_a Z_b / r phi(r / a_s), phi(x) = sum_k c_k exp(-d_k x) (the
// published universal screening function), enveloped by u(r / rc) of the
// edge's cutoff; half of it per ordered edge, in eV, not scaled by sigma_Z.
// Returns the edge's energy and dE/dr (float32 arithmetic; the reduction that
// uses them is float64).  zp = {k_e Z_a Z_b / 2, 1 / a_s} of the species pair.
__device__ __forceinline__ void zbl_edge(float r, float2 zp, float inv_rc, const BasisConst& bc, float& e,
                                         float& dedr) {
  const float y = r * inv_rc;
  if (!(y < 1.0f) || !(r > 0.0f)) {
    e = 0.0f;
    dedr = 0.0f;
    return;
  }
  const float cz[4] = {0.18175f, 0.50986f, 0.28022f, 0.02817f};
  const float dz[4] = {3.19980f, 0.94229f, 0.40290f, 0.20162f};
  const float x = r * zp.y;
  float phi = 0.0f, dphi = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float t = cz[k] * expf(-dz[k] * x);
    phi += t;
    dphi -= dz[k] * t;
  }
  const float yp1 = ipow(y, bc.p - 1), yp = yp1 * y;
  const float u = 1.0f - bc.c0 * yp + bc.c1 * yp * y - bc.c2 * yp * y * y;
  const float du = (-(float)bc.p * bc.c0 * yp1 + (float)(bc.p + 1) * bc.c1 * yp - (float)(bc.p + 2) * bc.c2 * yp * y) *
                   inv_rc;
  const float ir = 1.0f / r;
  const float a = zp.x * ir;                     // k_e Z_a Z_b / (2 r)
  e = a * phi * u;
  dedr = a * (dphi * zp.y * u + phi * du - phi * u * ir);
}

// Per atom i (float64): Etilde_i = sigma_Z E_i + mu_Z with E_i = sum_{row i} E_ij;
// F_i = sum_{e in row i} g_e - sum_{e with j_e = i} g_e  (g_e = dE/dd_e);
// per-atom virial W_i = - sum_{e in row i} d_e (x) g_e; with the ZBL term its energy
// joins Etilde_i and its dE/dd joins g_e in both gathers.
__global__ void atom_reduce_kernel(int n, int n_centres, const int* __restrict__ row_ptr, const int* __restrict__ col_ptr,
                                   const int* __restrict__ col_edge, const float* __restrict__ Ee,
                                   const float* __restrict__ g, const double* __restrict__ ed,
                                   const int* __restrict__ species, const double* __restrict__ sigma,
                                   const double* __restrict__ mu, bool want_forces, double* __restrict__ E_atom,
                                   double* __restrict__ F, double* __restrict__ Wat, const int* __restrict__ ei,
                                   const int* __restrict__ ej, const float2* __restrict__ zbl, BasisConst bc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = row_ptr[i], e1 = row_ptr[i + 1];
  const int z = species[i];
  double Ei = 0.0, Ez = 0.0;
  double f[3] = {0, 0, 0};
  double W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int e = b; e < e1; ++e) {
    Ei += (double)Ee[e];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    if (want_forces) {
      gx = g[3 * (size_t)e]; gy = g[3 * (size_t)e + 1]; gz = g[3 * (size_t)e + 2];
    }
    const double d0 = ed[3 * (size_t)e], d1 = ed[3 * (size_t)e + 1], d2 = ed[3 * (size_t)e + 2];
    if (zbl) {
      const int zj = species[ej[e]];
      const float r = (float)sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      float ez, dedr;
      zbl_edge(r, zbl[z * bc.ns + zj], pair_basis(bc, z, zj).x, bc, ez, dedr);
      Ez += (double)ez;
      const double s = (double)(dedr / r);
      gx += s * d0; gy += s * d1; gz += s * d2;
    }
    if (want_forces) {
      f[0] += gx; f[1] += gy; f[2] += gz;
      W[0] -= d0 * gx; W[1] -= d0 * gy; W[2] -= d0 * gz;
      W[3] -= d1 * gx; W[4] -= d1 * gy; W[5] -= d1 * gz;
      W[6] -= d2 * gx; W[7] -= d2 * gy; W[8] -= d2 * gz;
    }
  }
  E_atom[i] = (i < n_centres) ? sigma[z] * Ei + mu[z] + Ez : 0.0;
  if (want_forces) {
    for (int k = col_ptr[i]; k < col_ptr[i + 1]; ++k) {
      size_t e = (size_t)col_edge[k];
      double gx = g[3 * e], gy = g[3 * e + 1], gz = g[3 * e + 2];
      if (zbl) {   // the ZBL part of this edge's dE/dd (edge (k -> i): centre species first)
        const double d0 = ed[3 * e], d1 = ed[3 * e + 1], d2 = ed[3 * e + 2];
        const int zc = species[ei[e]];
        const float r = (float)sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        float ez, dedr;
        zbl_edge(r, zbl[zc * bc.ns + z], pair_basis(bc, zc, z).x, bc, ez, dedr);
        const double s = (double)(dedr / r);
        gx += s * d0; gy += s * d1; gz += s * d2;
      }
      f[0] -= gx; f[1] -= gy; f[2] -= gz;
    }
    F[3 * (size_t)i] = f[0]; F[3 * (size_t)i + 1] = f[1]; F[3 * (size_t)i + 2] = f[2];
    for (int q = 0; q < 9; ++q) Wat[9 * (size_t)i + q] = W[q];
  }
}

void atom_reduce(int n, int n_centres, const int* row_ptr, const int* col_ptr, const int* col_edge, const float* Ee,
                 const float* g, const double* ed, const int* species, const double* sigma, const double* mu,
                 bool want_forces, double* E_atom, double* F, double* Wat, const int* ei, const int* ej,
                 const Arch& a, cudaStream_t st) {
  if (n <= 0) return;
  atom_reduce_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, n_centres, row_ptr, col_ptr, col_edge, Ee, g, ed, species, sigma,
                                                      mu, want_forces, E_atom, F, Wat, ei, ej,
                                                      reinterpret_cast<const float2*>(a.zbl), make_basis(a));
}

// One block per structure: E_b = sum of its atoms' Etilde_i, W_b = sum of W_i
// (fixed-order tree reduction, so results are bitwise reproducible).  Also
// flags non-finite per-atom energies or forces.
__global__ void struct_reduce_kernel(const int64_t* __restrict__ offs, const double* __restrict__ E_atom,
                                     const double* __restrict__ Wat, const double* __restrict__ F, bool want_w,
                                     double* __restrict__ E_out, double* __restrict__ W_out,
                                     int* __restrict__ d_err) {
  const int b = blockIdx.x;
  const long long a0 = offs[b], a1 = offs[b + 1];
  __shared__ double sh[10][256];
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  bool bad = false;
  for (long long i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    double e = E_atom[i];
    acc[0] += e;
    bad |= !isfinite(e);
    if (want_w) {
      for (int q = 0; q < 9; ++q) acc[1 + q] += Wat[9 * i + q];
      bad |= !(isfinite(F[3 * i]) && isfinite(F[3 * i + 1]) && isfinite(F[3 * i + 2]));
    }
  }
  if (bad) atomicOr(d_err, kErrNonFinite);
  for (int q = 0; q < 10; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 10; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    E_out[b] = sh[0][0];
    if (want_w)
      for (int q = 0; q < 9; ++q) W_out[9 * b + q] = sh[1 + q][0];
  }
}

// Large single structures: first a fixed grid of blocks reduces contiguous
// atom ranges into partials (offsets describe the ranges), then one block
// reduces the partials; both in fixed order.
__global__ void partial_offsets_kernel(const int64_t* __restrict__ offs, int parts, int64_t* __restrict__ po) {
  const long long n = offs[1];
  for (int p = threadIdx.x; p <= parts; p += blockDim.x) po[p] = (n * p) / parts;
}

__global__ void sum_partials_kernel(const double* __restrict__ partE, const double* __restrict__ partW, int parts,
                                    bool want_w, double* __restrict__ E_out, double* __restrict__ W_out) {
  __shared__ double sh[10][256];
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = threadIdx.x; p < parts; p += blockDim.x) {
    acc[0] += partE[p];
    if (want_w)
      for (int q = 0; q < 9; ++q) acc[1 + q] += partW[9 * (size_t)p + q];
  }
  for (int q = 0; q < 10; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 10; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    E_out[0] = sh[0][0];
    if (want_w)
      for (int q = 0; q < 9; ++q) W_out[q] = sh[1 + q][0];
  }
}

void struct_reduce(int nstruct, const int64_t* offs, const double* E_atom, const double* Wat, const double* F,
                   bool want_w, double* E_out, double* W_out, int* d_err, double* scratch, int64_t n_atoms,
                   cudaStream_t st) {
  if (nstruct <= 0) return;
  const int parts = 1024;
  if (nstruct == 1 && n_atoms > 16 * parts && scratch) {
    int64_t* po = reinterpret_cast<int64_t*>(scratch);
    double* pE = scratch + (parts + 2);
    double* pW = pE + parts;
    partial_offsets_kernel<<<1, 256, 0, st>>>(offs, parts, po);
    struct_reduce_kernel<<<parts, 256, 0, st>>>(po, E_atom, Wat, F, want_w, pE, pW, d_err);
    sum_partials_kernel<<<1, 256, 0, st>>>(pE, pW, parts, want_w, E_out, W_out);
    return;
  }
  struct_reduce_kernel<<<nstruct, 256, 0, st>>>(offs, E_atom, Wat, F, want_w, E_out, W_out, d_err);
}

}  // namespace alg

namespace alg {

// ---------------------------------------------------------------------------
// Velocity Verlet (Sec. "Problem Overview": MD integrates Newton's equations
// with femtosecond steps).  Units: A, A/fs, amu, eV/A; kACC converts
// eV/(A amu) to A/fs^2.
// ---------------------------------------------------------------------------
constexpr double kACC = 9.648533212e-3;

__global__ void inv_mass_kernel(int n, const int* __restrict__ types, const double* __restrict__ masses, int nm,
                                double* __restrict__ inv_m, int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = types[i];
  const double m = (t >= 0 && t < nm) ? masses[t] : 0.0;
  if (!(m > 0)) atomicOr(err, kErrBadInput);
  inv_m[i] = (m > 0) ? 1.0 / m : 0.0;
}

// v += dt/2 a;  and, when drift, x += dt v
__global__ void kick_drift_kernel(int n, double* __restrict__ pos, double* __restrict__ vel,
                                  const double* __restrict__ F, const double* __restrict__ inv_m, double dt,
                                  bool drift) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double h = 0.5 * dt * kACC * inv_m[i];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    double v = vel[3 * (size_t)i + x] + h * F[3 * (size_t)i + x];
    vel[3 * (size_t)i + x] = v;
    if (drift) pos[3 * (size_t)i + x] += dt * v;
  }
}

// Kinetic energy 0.5 sum m v^2 / kACC in float64, two fixed-order levels.
__global__ void kinetic_partial_kernel(int n, const double* __restrict__ vel, const double* __restrict__ inv_m,
                                       double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double vx = vel[3 * (size_t)i], vy = vel[3 * (size_t)i + 1], vz = vel[3 * (size_t)i + 2];
    acc += (vx * vx + vy * vy + vz * vz) / inv_m[i];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void kinetic_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) acc += part[p];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * sh[0] / kACC;
}

void md_inv_mass(int n, const int* types, const double* masses, int nm, double* inv_m, int* err, cudaStream_t st) {
  if (n > 0) inv_mass_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, types, masses, nm, inv_m, err);
}

void md_kick(int n, double* pos, double* vel, const double* F, const double* inv_m, double dt, bool drift,
             cudaStream_t st) {
  if (n > 0) kick_drift_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, pos, vel, F, inv_m, dt, drift);
}

void md_kinetic(int n, const double* vel, const double* inv_m, double* part, double* out, cudaStream_t st) {
  const int parts = 256;
  kinetic_partial_kernel<<<parts, 256, 0, st>>>(n, vel, inv_m, part);
  kinetic_final_kernel<<<1, 256, 0, st>>>(part, parts, out);
}

}  // namespace alg
