// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M x N] = A[M x K] B^T,  A = edge activations (bf16, row-major, K contiguous),
//   B = weights (bf16, [N][K], K contiguous), float32 accumulation in TMEM,
// with the epilogues of epilogue.cuh (SiLU forward with pre-activation store,
// float32 output with addend, SiLU adjoint).  These are the MLP GEMMs of the
// two-body, latent and embedding/env-weight maps (Sec. "Mixed-precision
// calculations": matrix multiplications carry most of the cost).
//
// One CTA computes a 128 x BN tile: warp 0 issues TMA loads of 128 x 64 (A)
// and BN x 64 (B) bf16 tiles into a STAGES-deep shared-memory ring (128-byte
// swizzle), warp 1 allocates BN TMEM columns and issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = BN, K = 16 per instruction)
// from one thread, committing each stage back to the producer through an
// mbarrier; warps 2-5 read the accumulator with tcgen05.ld (each warp its
// 32-lane quarter of TMEM) and run the epilogue.  Every mbarrier wait is
// bounded (clock64 limit); on expiry the kernel sets the error word and
// unwinds (the host reports ALLEGRO_E_TIMEOUT).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "epilogue.cuh"
#include "internal.h"

namespace alg {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool gemm_tc_init(std::string* why) {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    if (why) *why = "cuTensorMapEncodeTiled entry point not available";
    return false;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

// 2-D bf16 tensor map: `inner` contiguous elements per row, `outer` rows,
// rows `row_bytes` apart; box box_inner x box_outer, 128-byte swizzle,
// out-of-bounds elements read as zero.
static bool make_tmap(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                      uint32_t box_inner, uint32_t box_outer) {
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait (about 2^32 SM cycles, ~2 s): false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > (1ll << 32)) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 consecutive 32-bit TMEM columns -> 32 registers per thread.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand tile written by TMA with
// the 128-byte swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);     // start address (bits 0-13)
  d |= (uint64_t)1 << 16;                        // leading-dimension byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride-dimension byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                        // swizzle mode: 128-byte
  return d;
}

// Instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, M = 128, N = BN.
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

constexpr int kTcBM = 128, kTcBK = 64;

template <int BN>
__host__ __device__ constexpr int tc_stages() {
  return (110 * 1024) / (kTcBM * kTcBK * 2 + BN * kTcBK * 2) < 2   ? 2
         : (110 * 1024) / (kTcBM * kTcBK * 2 + BN * kTcBK * 2) > 4 ? 4
                                                                    : (110 * 1024) / (kTcBM * kTcBK * 2 + BN * kTcBK * 2);
}

template <int BN>
__host__ __device__ constexpr int tc_tmem_cols() {
  return BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
}

template <int BN>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return (size_t)tc_stages<BN>() * (kTcBM * kTcBK * 2 + BN * kTcBK * 2) + 1024 + 256;
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiParams ep,
                   int M, int N, int K, int* __restrict__ err) {
  constexpr int STAGES = tc_stages<BN>();
  constexpr uint32_t A_BYTES = kTcBM * kTcBK * 2;
  constexpr uint32_t B_BYTES = BN * kTcBK * 2;
  constexpr uint32_t TMEM_COLS = tc_tmem_cols<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tfull + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * BN;
  const int nk = (K + kTcBK - 1) / kTcBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tc_alloc(tslot, TMEM_COLS);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], (r - 1) & 1)) {
          atomicOr(err, kErrTimeout);
          break;
        }
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sA + s * A_BYTES, &tmA, &full[s], kb * kTcBK, m0);
        tma_load_2d(sB + s * B_BYTES, &tmB, &full[s], kb * kTcBK, n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES, r = kb / STAGES;
        if (!mbar_wait(&full[s], r & 1)) {
          atomicOr(err, kErrTimeout);
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(sA + s * A_BYTES), b_addr = smem_u32(sB + s * B_BYTES);
#pragma unroll
        for (int k = 0; k < kTcBK / 16; ++k) {
          tc_mma(tmem, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32), idesc,
                 (kb > 0 || k > 0) ? 1u : 0u);
        }
        tc_commit(&empty[s]);
      }
      tc_commit(tfull);
    }
    __syncwarp();
  } else {
    const int q = warp & 3;   // TMEM lane quarter this warp may access
    const bool ok = mbar_wait(tfull, 0);
    if (!ok && lane == 0) atomicOr(err, kErrTimeout);
    tc_fence_after();
    if (ok) {
      const int m = m0 + q * 32 + lane;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;
        float v[32];
        tc_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (m < M) {
          if (ep.vec && n0 + c0 + 32 <= N) {
            epi_apply_vec32_bf16(ep, m, n0 + c0, v);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = n0 + c0 + j;
              if (n < N) epi_apply<bf16>(ep, m, n, v[j]);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, TMEM_COLS);
  }
}

template <int BN>
static bool launch_bn(const GemmArgs& g, const bf16* B, int ldb, cudaStream_t st, int* d_err, std::string* why) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes<BN>());
    if (e != cudaSuccess) {
      if (why) *why = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
      return false;
    }
    attr_set = true;
  }
  CUtensorMap ta, tb;
  if (!make_tmap(&ta, g.A, (uint64_t)g.K, (uint64_t)g.M, (uint64_t)g.lda * 2, kTcBK, kTcBM) ||
      !make_tmap(&tb, B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)ldb * 2, kTcBK, BN)) {
    if (why) *why = "cuTensorMapEncodeTiled failed (alignment or extent)";
    return false;
  }
  dim3 grid((g.M + kTcBM - 1) / kTcBM, (g.N + BN - 1) / BN);
  gemm_tc_kernel<BN><<<grid, 192, tc_smem_bytes<BN>(), st>>>(ta, tb, make_epi(g), g.M, g.N, g.K, d_err);
  return true;
}

bool gemm_tc_bf16(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why) {
  if (g.M <= 0 || g.N <= 0) return true;
  if (!gemm_tc_init(why)) return false;
  const bf16* B = g.trans ? g.W->b16T : g.W->b16;
  const int ldb = g.trans ? g.W->ldT : g.W->ld;
  if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (g.lda % 8) ||
      (ldb % 8)) {
    if (why) *why = "tcgen05 GEMM operands must be 16-byte aligned with pitches a multiple of 8 elements";
    return false;
  }
  const int tiles = (g.N + 255) / 256;
  int bn = (g.N + tiles - 1) / tiles;
  bn = (bn + 31) / 32 * 32;
  switch (bn) {
    case 32: return launch_bn<32>(g, B, ldb, st, d_err, why);
    case 64: return launch_bn<64>(g, B, ldb, st, d_err, why);
    case 96: return launch_bn<96>(g, B, ldb, st, d_err, why);
    case 128: return launch_bn<128>(g, B, ldb, st, d_err, why);
    case 160: return launch_bn<160>(g, B, ldb, st, d_err, why);
    case 192: return launch_bn<192>(g, B, ldb, st, d_err, why);
    case 224: return launch_bn<224>(g, B, ldb, st, d_err, why);
    default: return launch_bn<256>(g, B, ldb, st, d_err, why);
  }
}

}  // namespace alg
