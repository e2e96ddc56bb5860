// FP8 GEMMs on the 5th-generation tensor cores (tcgen05.mma kind::f8f6f4) for
// ALLEGRO_PREC_FP8 (the stretch precision of Sec. "Mixed-precision
// calculations": the MLP matrix multiplications at a lower operand precision,
// float32 accumulation):
//   C[M x N] = sA sB (QA QB^T),  QA = e4m3(A / sA),  QB = e4m3(B / sB),
// A = edge activations (bf16 in HBM, [M][lda], K contiguous, optionally the
// K-concatenation [A | A2]), B = weights pre-quantised to E4M3 ([N][ldb] bytes,
// K contiguous), sA and sB per-tensor powers of two.
//
// Per-tensor scaling ("current" scaling): every kernel that writes an
// activation which a later FP8 GEMM reads records max|value| of what it wrote
// into an amax slot (float bits, atomicMax); the GEMM reads its operand's slot
// at launch and takes sA = 2^ceil(log2(amax / 224)), so the largest element
// maps to at most half the E4M3 maximum (448) and no element saturates.  The
// weights' sB = 2^ceil(log2(max|W| / 448)) is fixed when the model is loaded.
// Both scales are powers of two, so scaling is exact and only the E4M3
// rounding (3 mantissa bits) remains.
//
// gemm_fp8_kernel<BN>: persistent, one CTA per SM walking 128 x BN tiles.
//   warp 0      TMA: B k-blocks (BN rows x 128 E4M3 bytes) into the operand
//               ring, A k-blocks as two 128 x 64 bf16 halves into a staging ring
//   warp 1      TMEM (two BN-column accumulators), tcgen05.mma kind::f8f6f4
//               (M = 128, N = BN, K = 32 per instruction) from one thread
//   warps 2-9   epilogue: tcgen05.ld, times sA sB, the float32/bf16 epilogue,
//               16-byte row stores, the output's amax
//   warps 10-13 converters: each staging half -> E4M3 (times 1/sA) into the
//               operand ring's A slot in the 128-byte-swizzled K-major layout
//               the tensor core reads (16 E4M3 per 16-byte unit, unit u of
//               row r at u ^ (r mod 8))
// Every mbarrier wait is bounded; on expiry the kernel sets the error word and
// unwinds (the host reports ALLEGRO_E_TIMEOUT).
#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "amax.cuh"
#include "epilogue.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace alg {

constexpr int kF8BK = 128;                          // E4M3 elements per operand k-block (one 128-byte row)
constexpr int kF8Stages = 3;                        // operand ring depth (k-blocks)
constexpr int kF8Stg = 4;                           // bf16 staging ring depth (64-column halves)
constexpr int kF8EpiWarps = 8;
constexpr int kF8ConvWarps = 4;
constexpr int kF8ConvWarp0 = 2 + kF8EpiWarps;      // first converter warp
constexpr int kF8Threads = 32 * (kF8ConvWarp0 + kF8ConvWarps);
constexpr uint32_t kF8ABytes = 128 * kF8BK;         // one E4M3 A k-block
constexpr uint32_t kF8StgBytes = 128 * 64 * 2;      // one bf16 staging half
constexpr float kF8Target = 224.0f;                 // largest |A| / sA (half of the E4M3 maximum 448)

template <int BN>
__host__ __device__ constexpr uint32_t f8_b_bytes() {
  return (uint32_t)BN * kF8BK;
}
template <int BN>
__host__ __device__ constexpr int f8_tmem_cols() {
  return BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
}
template <int BN>
__host__ __device__ constexpr int f8_smem_bytes() {
  return kF8Stages * (int)(kF8ABytes + f8_b_bytes<BN>()) + kF8Stg * (int)kF8StgBytes + 1024 + 1024;
}

// Instruction descriptor, kind::f8f6f4: D float32 (bits 4-5 = 1), A and B E4M3
// (format 0 in bits 7-9 and 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_e4m3() {
  return (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// sA = 2^ceil(log2(amax / 224)) and 1 / sA from an amax slot's float bits (1 when the
// tensor is all zero or not finite: the non-finite values then reach the outputs,
// where the host's finiteness check reports them)
__device__ __forceinline__ void f8_scale(unsigned bits, float& s, float& inv) {
  const float amax = __uint_as_float(bits);
  s = 1.0f;
  inv = 1.0f;
  if (!(amax > 0.0f) || !(amax < 3.0e38f)) return;
  int e;
  const float m = frexpf(amax / kF8Target, &e);   // amax / 224 = m 2^e, m in [0.5, 1)
  const int c = (m == 0.5f) ? e - 1 : e;
  s = ldexpf(1.0f, c);
  inv = ldexpf(1.0f, -c);
}

__device__ __forceinline__ unsigned f8_amax_bits(const unsigned* a, const unsigned* a2) {
  const unsigned x = a ? *a : 0u, y = a2 ? *a2 : 0u;
  return x > y ? x : y;
}

// sigmoid(z) = (1 + tanh(z / 2)) / 2 with the hardware tanh approximation (relative
// error ~2^-11, far below the E4M3 rounding of the products)
__device__ __forceinline__ float f8_sigmoid(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return fmaf(0.5f, t, 0.5f);
}

// 32 consecutive columns [n, n + 32) of row m (v already times sA sB): the epilogue of
// the bf16-storage path with plain stores; returns max|output| of an activation output
// (0 for the float32 output)
__device__ __forceinline__ float f8_epilogue(const EpiParams& ep, int m, int n, int N, float (&v)[32]) {
  const bool full = (n + 32 <= N) && ep.vec;
  if (ep.epi == EPI_F32) {
    float* o = reinterpret_cast<float*>(ep.out) + (size_t)m * ep.ldo + n;
    const float* a = ep.add ? reinterpret_cast<const float*>(ep.add) + (size_t)m * ep.ld_add + n : nullptr;
    if (full) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float4 x = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        if (a) {
          const float4 y = reinterpret_cast<const float4*>(a)[k];
          x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
        }
        reinterpret_cast<float4*>(o)[k] = x;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (n + j < N) o[j] = v[j] + (a ? a[j] : 0.0f);
    }
    return 0.0f;
  }
  if (ep.epi == EPI_FWD_SILU) {
    if (ep.pre) {
      bf16* pp = reinterpret_cast<bf16*>(ep.pre) + (size_t)m * ep.ldp + n;
      if (full) {
        store_bf16x32(pp, v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (n + j < N) pp[j] = __float2bfloat16_rn(v[j]);
      }
    }
    const float rs = ep.rowscale ? ep.rowscale[m] : 1.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = v[j] * f8_sigmoid(v[j]) * rs;
  } else if (ep.epi == EPI_BWD_SILU) {
    const bf16* zp = reinterpret_cast<const bf16*>(ep.pre) + (size_t)m * ep.ldp + n;
    float z[32];
    if (full) {
      load_bf16x32(zp, z);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = (n + j < N) ? __bfloat162float(zp[j]) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float sg = f8_sigmoid(z[j]);
      v[j] = v[j] * sg * (1.0f + z[j] * (1.0f - sg));
    }
  }
  bf16* o = reinterpret_cast<bf16*>(ep.out) + (size_t)m * ep.ldo + n;
  float amax = 0.0f;
  if (full) {
    store_bf16x32(o, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) amax = fmaxf(amax, fabsf(v[j]));
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (n + j < N) {
        o[j] = __float2bfloat16_rn(v[j]);
        amax = fmaxf(amax, fabsf(v[j]));
      }
  }
  return amax;
}

// 16 bf16 (two 16-byte units) times inv -> 16 E4M3 bytes (element k in byte k)
__device__ __forceinline__ uint4 f8_convert16(uint4 lo, uint4 hi, float inv) {
  const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
  uint32_t o[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[2 * p]));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[2 * p + 1]));
    const uint32_t qa = __nv_cvt_float2_to_fp8x2(make_float2(a.x * inv, a.y * inv), __NV_SATFINITE, __NV_E4M3);
    const uint32_t qb = __nv_cvt_float2_to_fp8x2(make_float2(b.x * inv, b.y * inv), __NV_SATFINITE, __NV_E4M3);
    o[p] = (qa & 0xFFFFu) | (qb << 16);
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ void fence_async_smem_f8() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct F8Params {
  int M, N, K, K1;              // A columns [0, K1) from tmA, [K1, K) from tmA2
  float sB;                     // the weights' scale
  const unsigned* amax_a;       // amax slots of A and A2 (float bits)
  const unsigned* amax_a2;
  unsigned* amax_out;           // this GEMM's output amax slot (or null)
  int* err;
};

template <int BN>
__global__ void __launch_bounds__(kF8Threads, 1)
    gemm_fp8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
                    const __grid_constant__ CUtensorMap tmB, EpiParams ep, F8Params fp) {
  constexpr uint32_t B_BYTES = f8_b_bytes<BN>();
  constexpr uint32_t COLS = f8_tmem_cols<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                                  // [kF8Stages] E4M3 A k-blocks
  uint8_t* sB = sA + kF8Stages * kF8ABytes;            // [kF8Stages] E4M3 B k-blocks
  uint8_t* sS = sB + kF8Stages * B_BYTES;              // [kF8Stg] bf16 staging halves
  uint64_t* full = reinterpret_cast<uint64_t*>(sS + kF8Stg * kF8StgBytes);   // B landed
  uint64_t* afull = full + kF8Stages;                  // A converted (one arrival per converter warp)
  uint64_t* empty = afull + kF8Stages;                 // the MMAs of the stage are complete
  uint64_t* sfull = empty + kF8Stages;                 // staging half landed
  uint64_t* sempty = sfull + kF8Stg;                   // staging half read (one arrival per converter warp)
  uint64_t* tfull = sempty + kF8Stg;                   // [2] accumulator ready
  uint64_t* tempty = tfull + 2;                        // [2] accumulator drained (one arrival per epilogue warp)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = fp.M, N = fp.N, K = fp.K;
  const int nk = (K + kF8BK - 1) / kF8BK;
  const int tiles_n = (N + BN - 1) / BN;
  const int ntiles = ((M + 127) / 128) * tiles_n;
  // tile t -> (row block t / tiles_n, column block t % tiles_n): the column blocks of a row
  // block run on neighbouring CTAs, so their A rows come from L2 after the first read
  auto tm0 = [&](int tt) { return (tt / tiles_n) * 128; };
  auto tn0 = [&](int tt) { return (tt % tiles_n) * BN; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kF8Stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&afull[s], kF8ConvWarps);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kF8Stg; ++s) {
      mbar_init(&sfull[s], 1);
      mbar_init(&sempty[s], kF8ConvWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kF8EpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tc_alloc(tslot, 2 * COLS);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;   // global k-block counter
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok && !*abort_flag; t += gridDim.x) {
        const int m0 = tm0(t), n0 = tn0(t);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const uint32_t s = g % kF8Stages, r = g / kF8Stages;
          if (g >= (uint32_t)kF8Stages && !mbar_wait(&empty[s], (r - 1) & 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], B_BYTES);
          tma_load_2d(sB + s * B_BYTES, &tmB, &full[s], kb * kF8BK, n0);
          for (int h = 0; h < 2 && ok; ++h) {
            const uint32_t g2 = 2 * g + h, s2 = g2 % kF8Stg, r2 = g2 / kF8Stg;
            if (g2 >= (uint32_t)kF8Stg && !mbar_wait(&sempty[s2], (r2 - 1) & 1)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&sfull[s2], kF8StgBytes);
            // first column of this half: A1 below K1, A2 up to K, past K (read as zero) from A1's map
            const int kc = kb * kF8BK + 64 * h;
            if (kc < fp.K1 || kc >= K) tma_load_2d(sS + s2 * kF8StgBytes, &tmA, &sfull[s2], kc, m0);
            else tma_load_2d(sS + s2 * kF8StgBytes, &tmA2, &sfull[s2], kc - fp.K1, m0);
          }
          if (!ok) break;
        }
      }
      if (!ok) {
        atomicOr(fp.err, kErrTimeout);
        *abort_flag = 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_e4m3<BN>();
      uint32_t g = 0;
      int lt = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
        const int b = lt & 1, use = lt >> 1;
        bool ok = !*abort_flag && mbar_wait(&tempty[b], (use & 1) ^ 1);
        if (ok) {
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * COLS);
          for (int kb = 0; kb < nk; ++kb, ++g) {
            const uint32_t s = g % kF8Stages, r = g / kF8Stages;
            if (!mbar_wait(&full[s], r & 1) || !mbar_wait(&afull[s], r & 1)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sA + s * kF8ABytes), b_addr = smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int k = 0; k < kF8BK / 32; ++k)   // 32 E4M3 = 32 bytes per instruction
              tc_mma_f8(dt, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32), idesc,
                        (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
          }
        }
        if (!ok) {
          atomicOr(fp.err, kErrTimeout);
          *abort_flag = 1;
        }
        tc_commit(&tfull[b]);
        if (!ok) break;
      }
    }
    __syncwarp();
  } else if (warp < kF8ConvWarp0) {
    // epilogue: 2 warps per TMEM lane quarter, alternating 32-column chunks
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    float scA, invA;
    f8_scale(f8_amax_bits(fp.amax_a, fp.amax_a2), scA, invA);
    const float sab = scA * fp.sB;
    float amx = 0.0f;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int b = lt & 1, use = lt >> 1;
      if (!mbar_wait(&tfull[b], use & 1)) {
        if (lane == 0) atomicOr(fp.err, kErrTimeout);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (*abort_flag) break;
      const int m0 = tm0(t), n0 = tn0(t);
      const int m = m0 + q * 32 + lane;
      const uint32_t base = tmem + (uint32_t)(b * COLS) + ((uint32_t)(q * 32) << 16);
      const int nch = (min(BN, N - n0) + 31) / 32;
      for (int c = h; c < nch; c += 2) {
        float v[32];
        tc_ld32(base + (uint32_t)(32 * c), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= sab;
        if (m < M) amx = fmaxf(amx, f8_epilogue(ep, m, n0 + 32 * c, N, v));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
    record_amax(fp.amax_out, amx);
  } else {
    // converters: staging halves (bf16, 128-byte swizzle: 8-element unit u of row r at
    // u ^ (r mod 8)) -> E4M3 A k-block (16-element unit u of row r at u ^ (r mod 8))
    const int ct = threadIdx.x - 32 * kF8ConvWarp0;   // 0..127
    float scA, invA;
    f8_scale(f8_amax_bits(fp.amax_a, fp.amax_a2), scA, invA);
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const uint32_t s = g % kF8Stages, r = g / kF8Stages;
        if (*abort_flag || (g >= (uint32_t)kF8Stages && !mbar_wait(&empty[s], (r - 1) & 1))) {
          ok = false;
          break;
        }
        uint8_t* a8 = sA + s * kF8ABytes;
        for (int h = 0; h < 2; ++h) {
          const uint32_t g2 = 2 * g + h, s2 = g2 % kF8Stg, r2 = g2 / kF8Stg;
          if (!mbar_wait(&sfull[s2], r2 & 1)) {
            ok = false;
            break;
          }
          const uint8_t* stg = sS + s2 * kF8StgBytes;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            // item -> (row, unit): eight consecutive lanes take eight consecutive rows of one
            // unit, so their 16-byte reads and writes fall on eight different bank groups
            const int it = ct + 128 * i;
            const int row = (it & 7) + 8 * (it >> 5), cc = (it >> 3) & 3, sw = row & 7;
            const uint4 lo = *reinterpret_cast<const uint4*>(stg + row * 128 + (((2 * cc) ^ sw) << 4));
            const uint4 hi = *reinterpret_cast<const uint4*>(stg + row * 128 + (((2 * cc + 1) ^ sw) << 4));
            *reinterpret_cast<uint4*>(a8 + row * 128 + (((4 * h + cc) ^ sw) << 4)) = f8_convert16(lo, hi, invA);
          }
          // the staging reads are ordered before the next TMA write into the half
          fence_async_smem_f8();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sempty[s2]);
        }
        if (!ok) break;
        // the A tile's generic-proxy writes become visible to the tensor core
        fence_async_smem_f8();
        __syncwarp();
        if (lane == 0) mbar_arrive(&afull[s]);
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(fp.err, kErrTimeout);
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, 2 * COLS);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr int kF8MaxDevices = 64;

static int f8_device() {
  int d = 0;
  cudaGetDevice(&d);
  return (d >= 0 && d < kF8MaxDevices) ? d : 0;
}

template <int BN>
static bool launch_fp8(const GemmArgs& g, const uint8_t* B8, int ldb8, float sB, cudaStream_t st, int* d_err,
                       std::string* why) {
  static bool attr_set[kF8MaxDevices] = {};
  static int nsm[kF8MaxDevices] = {};
  constexpr int smem = f8_smem_bytes<BN>();
  static_assert(smem <= 232448, "FP8 GEMM shared memory");
  const int dev = f8_device();
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(gemm_fp8_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) {
      if (why) *why = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
      return false;
    }
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    nsm[dev] = n > 0 ? n : 148;
    attr_set[dev] = true;
  }
  const int K1 = g.A2 ? g.K1 : g.K;
  CUtensorMap ta, ta2, tb;
  bool ok = tc_tensor_map_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.A, (uint64_t)K1, (uint64_t)g.M,
                             (uint64_t)g.lda * 2, 64, 128) &&
            tc_tensor_map_2d(&ta2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.A2 ? g.A2 : g.A,
                             (uint64_t)(g.A2 ? g.K - K1 : K1), (uint64_t)g.M, (uint64_t)(g.A2 ? g.lda2 : g.lda) * 2,
                             64, 128) &&
            tc_tensor_map_2d(&tb, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, B8, (uint64_t)g.K, (uint64_t)g.N,
                             (uint64_t)ldb8, kF8BK, BN);
  if (!ok) {
    if (why) *why = "cuTensorMapEncodeTiled failed (FP8 GEMM operands)";
    return false;
  }
  F8Params fp;
  fp.M = g.M; fp.N = g.N; fp.K = g.K; fp.K1 = K1;
  fp.sB = sB;
  fp.amax_a = g.amax_a; fp.amax_a2 = g.A2 ? g.amax_a2 : nullptr;
  fp.amax_out = g.amax_out;
  fp.err = d_err;
  const int tiles = ((g.M + 127) / 128) * ((g.N + BN - 1) / BN);
  const int grid = tiles < nsm[dev] ? tiles : nsm[dev];
  gemm_fp8_kernel<BN><<<grid, kF8Threads, smem, st>>>(ta, ta2, tb, make_epi(g), fp);
  return true;
}

bool gemm_tc_fp8(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why) {
  if (g.M <= 0 || g.N <= 0) return true;
  if (!gemm_tc_init(why)) return false;
  if (!(g.epi == EPI_FWD_SILU || g.epi == EPI_F32 || g.epi == EPI_BWD_SILU || g.epi == EPI_LINEAR)) {
    if (why) *why = "FP8 GEMM: unsupported epilogue";
    return false;
  }
  if (!g.amax_a || (g.A2 && !g.amax_a2)) {
    if (why) *why = "FP8 GEMM: operand without an amax slot";
    return false;
  }
  const uint8_t* B = g.Bover8 ? g.Bover8 : (g.trans ? g.W->f8T : g.W->f8);
  const int ldb = g.Bover8 ? g.ldb_over8 : (g.trans ? g.W->ld8T : g.W->ld8);
  const float sB = g.Bover8 ? g.sBover8 : (g.trans ? g.W->s8T : g.W->s8);
  if (!B) {
    if (why) *why = "FP8 GEMM: no E4M3 copy of the weights";
    return false;
  }
  B += (size_t)g.b_row0 * ldb;
  if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (g.lda % 8) ||
      (ldb % 16) || (g.A2 && ((reinterpret_cast<uintptr_t>(g.A2) & 15) || (g.lda2 % 8) || (g.K1 % 64) ||
                             g.K1 <= 0 || g.K1 >= g.K))) {
    if (why) *why = "FP8 GEMM operands must be 16-byte aligned (A pitch a multiple of 8, B of 16 elements)";
    return false;
  }
  const int tiles = (g.N + 255) / 256;
  int bn = (g.N + tiles - 1) / tiles;
  bn = (bn + 31) / 32 * 32;
  switch (bn) {
    case 32: return launch_fp8<32>(g, B, ldb, sB, st, d_err, why);
    case 64: return launch_fp8<64>(g, B, ldb, sB, st, d_err, why);
    case 96: return launch_fp8<96>(g, B, ldb, sB, st, d_err, why);
    case 128: return launch_fp8<128>(g, B, ldb, sB, st, d_err, why);
    case 160: return launch_fp8<160>(g, B, ldb, sB, st, d_err, why);
    case 192: return launch_fp8<192>(g, B, ldb, sB, st, d_err, why);
    case 224: return launch_fp8<224>(g, B, ldb, sB, st, d_err, why);
    default: return launch_fp8<256>(g, B, ldb, sB, st, d_err, why);
  }
}

__global__ void quant_e4m3_kernel(const float* __restrict__ src, int rows, int cols, int lds,
                                  uint8_t* __restrict__ dst, int ldd, float inv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)rows * ldd) return;
  const int r = (int)(i / ldd), k = (int)(i - (long long)r * ldd);
  const float v = (k < cols) ? src[(size_t)r * lds + k] * inv : 0.0f;
  dst[i] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

void fp8_quantize(const float* src, int rows, int cols, int lds, uint8_t* dst, int ldd, float inv_scale,
                  cudaStream_t st) {
  const long long n = (long long)rows * ldd;
  if (n <= 0) return;
  quant_e4m3_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, rows, cols, lds, dst, ldd, inv_scale);
}

}  // namespace alg
