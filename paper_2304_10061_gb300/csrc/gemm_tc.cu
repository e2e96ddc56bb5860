// BF16 GEMMs on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M x N] = A[M x K] B^T,  A = edge activations (bf16, row-major, K contiguous),
//   B = weights (bf16, [N][K], K contiguous), float32 accumulation in TMEM,
// with fused epilogues (SiLU forward with pre-activation store, SiLU adjoint,
// the adjoint head of x = u silu(z), the last latent layer with the folded
// edge energy, linear / float32 outputs).  These are the MLP GEMMs of the
// two-body, latent and embedding/env-weight maps (Sec. "Mixed-precision
// calculations": matrix multiplications carry most of the cost).
//
// gemm_tc_kernel<BN, EPQ>: one layer.  Persistent: one CTA per SM walks 128 x BN
// tiles (the column blocks of a row block on neighbouring CTAs, so A rows are
// shared through L2).  Warp 0 issues TMA loads of 128 x 64 (A) and BN x 64 (B)
// bf16 tiles into a shared-memory ring (128-byte swizzle), warp 1 allocates
// two BN-column TMEM accumulators and issues tcgen05.mma.cta_group::1.kind::f16
// (M = 128, N = BN, K = 16 per instruction) from one thread, 4 x EPQ epilogue
// warps (EPQ per 32-lane TMEM quarter) drain the other accumulator with
// tcgen05.ld and write 32 x 32 boxes through shared memory with TMA stores.
//
// gemm_chain_pipe_kernel<N1, N2, E1, E2>: two consecutive layers with the
// intermediate activation kept on chip (described at the kernel).
//
// Every mbarrier wait is bounded (clock64 limit); on expiry the kernel sets the
// error word and unwinds (the host reports ALLEGRO_E_TIMEOUT).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "epilogue.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

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
// out-of-bounds elements read as zero.  L2 fills at 256-byte granularity when
// the map covers whole rows, at 64 bytes when it covers only part of each row
// of its array (the x columns of [x | s], 64 columns of a 256-wide buffer):
// larger fills would pull in the columns that are not read.
static bool make_tmap(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                      uint32_t box_inner, uint32_t box_outer) {
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        inner * 2 < row_bytes ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_tensor_map_2d(CUtensorMap* tm, CUtensorMapDataType dtype, int esize, const void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  if (!g_encode) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B,
                        inner * esize < row_bytes ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}


// Instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, M = 128, N = BN.
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

constexpr int kTcBM = 128, kTcBK = 64;
// Epilogue warps: EPQ per 32-lane TMEM quarter (2 or 4), warps 2 .. 2 + 4 EPQ - 1.
// Four per quarter for the arithmetic-heavy epilogues (more warps hide the
// latency of the TMEM loads and transcendental ops), two for the plain copies
// (which rather want the deeper operand ring and the double-buffered output
// staging that the smaller epilogue footprint leaves room for).
template <int EPQ> __host__ __device__ constexpr int tc_threads() { return 64 + 32 * 4 * EPQ; }
// Shared memory of one CTA: the operand ring (A and B k-blocks), then per
// epilogue warp its output staging buffers and its input slot, then the
// mbarriers, flags and partial row sums.  The epilogue part depends on the
// mode (TcLayout, chosen on the host): a bf16 32x32 output box is 2 KB, a
// float32 box or an activation + pre-activation pair 4 KB; two output buffers
// (double-buffered TMA stores) with two warps per quarter, one with four; an
// input slot of 2 KB per bf16 input (pre-activation, addend).  The ring takes
// the rest, up to kTcMaxStages k-blocks.
constexpr int kTcSmemMax = 232448;           // dynamic shared memory per block (227 KB)
constexpr int kTcMisc = 4096;                // mbarriers, TMEM slot, flags, partial row sums
constexpr int kTcMaxStages = 8;

struct TcLayout {
  int stages;      // operand ring depth
  int out_box;     // bytes per output buffer
  int n_out;       // output buffers per warp
  int in_slot;     // bytes of the input slot
  int epi_slot;    // n_out * out_box + in_slot
};

template <int BN>
__host__ __device__ constexpr int tc_stage_bytes() {
  return kTcBM * kTcBK * 2 + BN * kTcBK * 2;
}

template <int BN>
__host__ __device__ constexpr int tc_tmem_cols() {   // one accumulator buffer
  return BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
}

template <int BN, int EPQ>
static TcLayout tc_layout(int epi, bool pre) {
  TcLayout L;
  const bool wide_out = (epi == EPI_F32) || (epi == EPI_FWD_SILU && pre);
  L.out_box = wide_out ? 4096 : 2048;
  L.n_out = (EPQ == 2) ? 2 : 1;
  L.in_slot = (epi == EPI_BWD_SILU) ? 2048 : (epi == EPI_HEAD ? 4096 : 0);
  L.epi_slot = L.n_out * L.out_box + L.in_slot;
  const int epi_smem = 4 * EPQ * L.epi_slot;
  const int st = (kTcSmemMax - 1024 - kTcMisc - epi_smem) / tc_stage_bytes<BN>();
  L.stages = st > kTcMaxStages ? kTcMaxStages : st;
  return L;
}
template <int BN, int EPQ>
static size_t tc_smem_bytes(const TcLayout& L) {
  return (size_t)L.stages * tc_stage_bytes<BN>() + (size_t)4 * EPQ * L.epi_slot + 1024 + kTcMisc;
}

// --- epilogue staging: 32 x 32 boxes moved by TMA --------------------------
// bf16 box rows are 64 bytes (64-byte swizzle), float32 box rows 128 bytes
// (128-byte swizzle); the 16-byte unit u of row r sits at unit u ^ f(r) so the
// row-per-lane accesses spread over all banks.
__device__ __forceinline__ uint32_t sw64(int r, int u) { return r * 64 + ((u ^ ((r >> 1) & 3)) << 4); }
__device__ __forceinline__ uint32_t sw128(int r, int u) { return r * 128 + ((u ^ (r & 7)) << 4); }

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, const void* src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void st_bf16_row(uint8_t* box, int r, const float (&v)[32]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    uint4 x = make_uint4(pack_bf16x2(v[8 * u + 0], v[8 * u + 1]), pack_bf16x2(v[8 * u + 2], v[8 * u + 3]),
                         pack_bf16x2(v[8 * u + 4], v[8 * u + 5]), pack_bf16x2(v[8 * u + 6], v[8 * u + 7]));
    *reinterpret_cast<uint4*>(box + sw64(r, u)) = x;
  }
}
__device__ __forceinline__ void ld_bf16_row(const uint8_t* box, int r, float (&v)[32]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    uint4 x = *reinterpret_cast<const uint4*>(box + sw64(r, u));
    uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w[t]));
      v[8 * u + 2 * t] = f.x;
      v[8 * u + 2 * t + 1] = f.y;
    }
  }
}
__device__ __forceinline__ void st_f32_row(uint8_t* box, int r, const float (&v)[32]) {
#pragma unroll
  for (int u = 0; u < 8; ++u)
    *reinterpret_cast<float4*>(box + sw128(r, u)) = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
}
__device__ __forceinline__ void ld_f32_row(const uint8_t* box, int r, float (&v)[32]) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    float4 x = *reinterpret_cast<const float4*>(box + sw128(r, u));
    v[4 * u] = x.x; v[4 * u + 1] = x.y; v[4 * u + 2] = x.z; v[4 * u + 3] = x.w;
  }
}

// 16 columns (half hh of a 32-column box row) into the swizzled staging boxes.
__device__ __forceinline__ void st_bf16_half(uint8_t* box, int r, int hh, const float (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    uint4 x = make_uint4(pack_bf16x2(v[8 * u + 0], v[8 * u + 1]), pack_bf16x2(v[8 * u + 2], v[8 * u + 3]),
                         pack_bf16x2(v[8 * u + 4], v[8 * u + 5]), pack_bf16x2(v[8 * u + 6], v[8 * u + 7]));
    *reinterpret_cast<uint4*>(box + sw64(r, 2 * hh + u)) = x;
  }
}
__device__ __forceinline__ void st_f32_half(uint8_t* box, int r, int hh, const float (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<float4*>(box + sw128(r, 4 * hh + u)) = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
}
__device__ __forceinline__ void load_bf16x16(const bf16* p, float (&v)[16]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    uint4 x = q[k];
    uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w[t]));
      v[8 * k + 2 * t] = f.x;
      v[8 * k + 2 * t + 1] = f.y;
    }
  }
}

// sigma(z) = (1 + tanh(z / 2)) / 2 with the hardware tanh approximation (one
// transcendental-unit op instead of an exponential and a reciprocal; its
// relative error, about 2^-11, is below the bf16 rounding of the outputs)
__device__ __forceinline__ float fast_sigmoid(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return fmaf(0.5f, t, 0.5f);
}

// Column pairs in packed fp32 operations (FMUL2 / FFMA2, sm_100 and later);
// each half is the ordinary IEEE fp32 operation.
__device__ __forceinline__ float2 f2_bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// fast_sigmoid of both halves
__device__ __forceinline__ float2 fast_sigmoid2(float2 z) {
  const float2 h = f2_mul(f2_bc(0.5f), z);
  float tx, ty;
  asm("tanh.approx.f32 %0, %1;" : "=f"(tx) : "f"(h.x));
  asm("tanh.approx.f32 %0, %1;" : "=f"(ty) : "f"(h.y));
  return f2_fma(f2_bc(0.5f), make_float2(tx, ty), f2_bc(0.5f));
}
// silu'(z) / sigmoid(z) = 1 + z (1 - sigmoid(z)), from s = sigmoid(z)
__device__ __forceinline__ float2 dsilu_factor2(float2 z, float2 sg) {
  return f2_fma(z, f2_fma(sg, f2_bc(-1.0f), f2_bc(1.0f)), f2_bc(1.0f));
}
// elements (2k, 2k + 1) of a row of raw bf16 words
__device__ __forceinline__ float2 bf16_word_pair(uint32_t x) {
  return make_float2(__uint_as_float(x << 16), __uint_as_float(x & 0xffff0000u));
}

struct EpiMaps {
  CUtensorMap out, pre, add;
};

// Raw bf16 words of one 32-column row of a swizzled bf16 32x32 box (16 words).
__device__ __forceinline__ void ld_bf16_row_raw(const uint8_t* box, int r, uint32_t (&w)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const uint4 x = *reinterpret_cast<const uint4*>(box + sw64(r, u));
    w[4 * u] = x.x; w[4 * u + 1] = x.y; w[4 * u + 2] = x.z; w[4 * u + 3] = x.w;
  }
}
// element j (0..31) of such a row
__device__ __forceinline__ float bf16_word_elem(const uint32_t (&w)[16], int j) {
  const uint32_t x = w[j >> 1];
  return __uint_as_float((j & 1) ? (x & 0xffff0000u) : (x << 16));
}

// Persistent kernel: CTA b handles tiles b, b + gridDim.x, ...  Two TMEM
// accumulator buffers: the MMA warp fills buffer (t & 1) while the epilogue
// warps drain the other, and the TMA producer runs ahead through the
// shared-memory ring across tile boundaries.  EPQ (2 or 4) epilogue warps
// share each 32-lane quarter of TMEM (warp h takes the 32-column chunks h,
// h + EPQ, ...); per chunk a warp takes its epilogue inputs (pre-activation,
// addend; fetched by TMA one chunk ahead), computes in registers 16 columns
// at a time, stages the results in swizzled shared memory and writes them
// back with TMA bulk stores.  The head and last-layer modes combine a
// quarter's partial row sums in a fixed warp order.
// With 18 warps (EPQ = 4) five share one SM sub-partition's 16K registers: at
// most 96 per thread.
template <int BN, int EPQ>
__global__ void __launch_bounds__(tc_threads<EPQ>(), 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmB, const __grid_constant__ EpiMaps em, EpiParams ep,
                   TcLayout lay, int M, int N, int K, int K1, int* __restrict__ err) {
  const int STAGES = lay.stages;
  constexpr int kEpiWarps = 4 * EPQ;
  const int kEpiSlot = lay.epi_slot;
  const int kNOut = lay.n_out;
  constexpr uint32_t A_BYTES = kTcBM * kTcBK * 2;
  constexpr uint32_t B_BYTES = BN * kTcBK * 2;
  constexpr uint32_t COLS = tc_tmem_cols<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint8_t* sE = sB + STAGES * B_BYTES;                       // epilogue staging (1024-aligned)
  uint64_t* full = reinterpret_cast<uint64_t*>(sE + 4 * EPQ * kEpiSlot);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;     // [2]
  uint64_t* tempty = tfull + 2;         // [2]
  uint64_t* rsbar = tempty + 2;         // [4 quarters][2 buffers]: partial row sums ready
  uint64_t* inbar = rsbar + 8;          // [kEpiWarps]: input slot filled
  uint32_t* tslot = reinterpret_cast<uint32_t*>(inbar + kEpiWarps);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  float* rowpart = reinterpret_cast<float*>(tslot + 4);   // [4 quarters][2 buffers][EPQ - 1][32] partial row sums

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (K + kTcBK - 1) / kTcBK;
  const int tiles_m = (M + kTcBM - 1) / kTcBM, tiles_n = (N + BN - 1) / BN;
  const int ntiles = tiles_m * tiles_n;
  // tile t -> (row block t / tiles_n, column block t % tiles_n): the column
  // blocks of one row block run on neighbouring CTAs at the same time, so the
  // A rows they share come from L2 after the first read
  auto tm0 = [&](int tt) { return (tt / tiles_n) * kTcBM; };
  auto tn0 = [&](int tt) { return (tt % tiles_n) * BN; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    for (int q = 0; q < 8; ++q) mbar_init(&rsbar[q], EPQ - 1);
    for (int q = 0; q < kEpiWarps; ++q) mbar_init(&inbar[q], 1);
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
      uint32_t g = 0;   // global k-block counter (ring position)
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        const int m0 = tm0(t), n0 = tn0(t);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const uint32_t s = g % STAGES, r = g / STAGES;
          if (g >= (uint32_t)STAGES && !mbar_wait(&empty[s], (r - 1) & 1)) {
            atomicOr(err, kErrTimeout);
            *abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
          if (kb * kTcBK < K1) tma_load_2d(sA + s * A_BYTES, &tmA, &full[s], kb * kTcBK, m0);
          else tma_load_2d(sA + s * A_BYTES, &tmA2, &full[s], kb * kTcBK - K1, m0);   // columns of A2
          tma_load_2d(sB + s * B_BYTES, &tmB, &full[s], kb * kTcBK, n0);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      uint32_t g = 0;
      int lt = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
        const int b = lt & 1, use = lt >> 1;
        bool ok = !*abort_flag && mbar_wait(&tempty[b], (use & 1) ^ 1);
        if (ok) {
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * COLS);
          for (int kb = 0; kb < nk; ++kb, ++g) {
            const uint32_t s = g % STAGES, r = g / STAGES;
            if (!mbar_wait(&full[s], r & 1)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sA + s * A_BYTES), b_addr = smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int k = 0; k < kTcBK / 16; ++k)
              tc_mma(dt, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32), idesc,
                     (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
          }
        }
        if (!ok) {
          atomicOr(err, kErrTimeout);
          *abort_flag = 1;
        }
        tc_commit(&tfull[b]);
        if (!ok) break;
      }
    }
    __syncwarp();
  } else {
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int ew = warp - 2;           // epilogue warp index 0..kEpiWarps-1
    const int h = ew >> 2;             // 0..EPQ-1 within the quarter
    uint8_t* my_out = sE + ew * kEpiSlot;
    uint8_t* my_in = my_out + kNOut * lay.out_box;
    const bool need_pre = (ep.epi == EPI_BWD_SILU || ep.epi == EPI_HEAD);
    const bool need_add = (ep.add != nullptr) && (ep.epi == EPI_HEAD);
    const uint32_t in_bytes = (need_pre ? 2048u : 0u) + (need_add ? 2048u : 0u);
    const bool out_f32 = (ep.epi == EPI_F32);
    const bool store_pre = (ep.epi == EPI_FWD_SILU) && ep.pre;
    const bool rowsums = (ep.epi == EPI_HEAD || ep.epi == EPI_LAST);
    uint32_t in_par = 0;
    // fetch the inputs of chunk c of tile t into the slot (lane 0 issues)
    auto fetch = [&](int tt, int cc) {
      if (in_bytes == 0 || tt >= ntiles) return;
      if (lane == 0) {
        const int mb = tm0(tt) + q * 32, nb = tn0(tt) + 32 * cc;
        mbar_expect_tx(&inbar[ew], in_bytes);
        if (need_pre) tma_load_2d(my_in, &em.pre, &inbar[ew], nb, mb);
        if (need_add) tma_load_2d(my_in + 2048, &em.add, &inbar[ew], nb, mb);
      }
    };
    auto nch_of = [&](int tt) { return (min(BN, N - tn0(tt)) + 31) / 32; };
    int lt = 0;
    int oc = 0;                        // output chunks issued (buffer = oc % kNOut)
    if (h < nch_of(blockIdx.x)) fetch(blockIdx.x, h);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int b = lt & 1, use = lt >> 1;
      const bool ok = mbar_wait(&tfull[b], use & 1);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      if (*abort_flag) break;
      const int m0 = tm0(t), n0 = tn0(t);
      const int mrow = m0 + q * 32;     // first row of this warp's box
      const int m = mrow + lane;
      const bool live = m < M;
      const float rs = (live && ep.rowscale) ? ep.rowscale[m] : 1.0f;
      const float sg = (live && ep.rowsig) ? ep.rowsig[m] : 1.0f;
      float acc1 = 0.0f;
      const uint32_t base = tmem + (uint32_t)(b * COLS) + ((uint32_t)(q * 32) << 16);
      const int nch = nch_of(t);
      for (int c = h; c < nch; c += EPQ) {
        uint8_t* ob = my_out + (oc % kNOut) * lay.out_box;
        // inputs of this chunk, kept as packed bf16 words
        uint32_t zw[16], aw[16];
        if (in_bytes) {
          if (!mbar_wait(&inbar[ew], in_par)) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            *abort_flag = 1;
          }
          in_par ^= 1u;
          if (need_pre) ld_bf16_row_raw(my_in, lane, zw);
          if (need_add) ld_bf16_row_raw(my_in + 2048, lane, aw);
          // the slot's generic reads are ordered before the next TMA write into it
          fence_async_smem();
          __syncwarp();
          // prefetch this warp's next chunk (possibly in its next tile)
          if (c + EPQ < nch) fetch(t, c + EPQ);
          else if (t + (int)gridDim.x < ntiles && h < nch_of(t + gridDim.x)) fetch(t + gridDim.x, h);
        }
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int n = n0 + 32 * c + 16 * hh;
          float v[16];
          tc_ld16(base + (uint32_t)(32 * c + 16 * hh), v);
          float o2[16];
          if (ep.epi == EPI_FWD_SILU) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              o2[j] = v[j];
              v[j] = v[j] * fast_sigmoid(v[j]) * rs;
            }
          } else if (ep.epi == EPI_F32 || ep.epi == EPI_LINEAR) {
            // the accumulator as it is (float32 or activation type)
          } else if (ep.epi == EPI_BWD_SILU) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float z = bf16_word_elem(zw, 16 * hh + j);
              const float sgm = fast_sigmoid(z);
              v[j] = v[j] * sgm * (1.0f + z * (1.0f - sgm));
            }
          } else if (ep.epi == EPI_HEAD) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float z = bf16_word_elem(zw, 16 * hh + j);
              const float xb = v[j] + (need_add ? bf16_word_elem(aw, 16 * hh + j) : 0.0f);
              const float sgm = fast_sigmoid(z);
              acc1 += xb * z * sgm;
              v[j] = xb * rs * sgm * (1.0f + z * (1.0f - sgm));
            }
          } else {   // EPI_LAST
            // the 16 entries of v for these columns (one vector load each for 4 when all are inside N)
            float vv[16];
            if (n + 16 <= N) {
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(ep.v + n) + k4);
                vv[4 * k4] = x.x; vv[4 * k4 + 1] = x.y; vv[4 * k4 + 2] = x.z; vv[4 * k4 + 3] = x.w;
              }
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j) vv[j] = (n + j < N) ? ep.v[n + j] : 0.0f;
            }
            const float srs = sg * rs;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float sgm = fast_sigmoid(v[j]);
              acc1 += vv[j] * v[j] * sgm;
              v[j] = srs * vv[j] * sgm * (1.0f + v[j] * (1.0f - sgm));
            }
          }
          if (hh == 0) {
            // the staging buffer is free once the store that used it has read it
            if (lane == 0) {
              if (kNOut == 1) bulk_wait_read0();
              else bulk_wait_read1();
            }
            __syncwarp();
          }
          if (out_f32) st_f32_half(ob, lane, hh, v);
          else st_bf16_half(ob, lane, hh, v);
          if (store_pre) st_bf16_half(ob + 2048, lane, hh, o2);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&em.out, ob, n0 + 32 * c, mrow);
          if (store_pre) tma_store_2d(&em.pre, ob + 2048, n0 + 32 * c, mrow);
          bulk_commit();
        }
        ++oc;
      }
      // every TMEM read of this buffer by this warp is complete (tcgen05.ld waits)
      tc_fence_before();
      __syncwarp();
      if (!rowsums) {
        if (lane == 0) mbar_arrive(&tempty[b]);
      } else {
        // combine the quarter's partial row sums in a fixed order (h = 0, 1, 2, 3).
        // Warp h = 0 releases the TMEM buffer only after reading the partials,
        // so no warp can overwrite a partial slot (indexed by the buffer)
        // before it is read.
        auto part_of = [&](int hp) -> float* { return rowpart + (((q * 2 + b) * (EPQ - 1) + (hp - 1)) * 32); };
        float* part = h != 0 ? part_of(h) : nullptr;
        if (h != 0) {
          part[lane] = acc1;
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(&rsbar[q * 2 + b]);
            mbar_arrive(&tempty[b]);
          }
        } else {
          if (!mbar_wait(&rsbar[q * 2 + b], use & 1)) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            *abort_flag = 1;
          }
          float tot = acc1;
#pragma unroll
          for (int hp = 1; hp < EPQ; ++hp)
            tot += part_of(hp)[lane];
          if (live) {
            if (ep.epi == EPI_HEAD) {
              ep.ubar[m] += tot;
            } else {
              ep.Eout[m] = rs * tot;
              ep.ubar[m] = sg * tot;
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[b]);
        }
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, 2 * COLS);
  }
}

// ===========================================================================
// Pipelined chain (N1 = 128 or 256, N2 <= 256): C2 = epi2(epi1(A1 B1^T) B2^T)
// with the intermediate activation kept on chip.  GEMM 1 runs as NH = N1/128
// jobs of 128 output columns each, into a two-slot ring of 128-column TMEM
// accumulators (columns [0, 128) and [128, 256)); GEMM 2 accumulates in
// columns [256, 256 + N2).  Two epilogue warp groups run at the same time:
// group 1 (8 warps) drains each GEMM-1 job into its half of the swizzled A
// operand of GEMM 2 (on chip, never written to HBM), group 2 (8 warps) drains
// GEMM 2's accumulator to HBM.  GEMM 2 consumes its A operand half by half,
// each half released to group 1 as soon as its MMAs complete.  MMA job order:
//   NH = 1:  G1(0); per tile i: G1(i+1), G2(i)
//   NH = 2:  G1(0,a); per tile i: G1(i,b), G2(i,a), G1(i+1,a), G2(i,b)
//            or (late GEMM 2) G1(i,b), G1(i+1,a), G2(i,a), G2(i,b)
// so that the tensor pipe works on one job while group 1 drains the previous
// one.  The late order gives group 2 one more GEMM-1 job to drain GEMM 2 of
// tile i - 1 (GEMM 2 of tile i needs the single GEMM-2 accumulator back); it
// is used for the pairs it measured faster on (256-wide second layers after an
// adjoint head, the last latent layer, the adjoint -> linear pair).  The
// operand ring (3 stages of 32 KB) carries [A1 k-block | B1 rows of the job]
// for GEMM-1 jobs and B2 k-blocks for GEMM-2 halves, in job order.
// GEMM 1's A operand may be the K-concatenation [A1 | A1b] (split at K1a, a
// multiple of 64 columns).
//   epi1: FWD_SILU (pre-activation stored), HEAD (pre-activation loaded, row
//         sums added to ubar) or BWD_SILU (pre-activation loaded, the product
//         also stored to HBM);
//   epi2: FWD_SILU (pre-activation stored), LAST (the single GEMM's last-layer
//         epilogue), BWD_SILU (pre-activation loaded) or LINEAR.
// HEAD and LAST are not combined in one launch (they share the row-sum slot).
// ===========================================================================
constexpr int kCfWarps = 16;                       // 8 per epilogue group
constexpr int kCfThreads = 64 + 32 * kCfWarps;
constexpr int kCfStages = 3;
constexpr int kCfJobN = 128;                       // output columns of one GEMM-1 job

__host__ __device__ constexpr int cf_stage_bytes(int n1, int n2) {
  // the larger of [A1 k-block | 128 rows of B1] and [N2 rows of B2]
  return (kTcBM + kCfJobN) * kTcBK * 2 > n2 * kTcBK * 2 ? (kTcBM + kCfJobN) * kTcBK * 2 : n2 * kTcBK * 2;
}
// group-2 staging buffers per warp: two when shared memory allows, one for 256-wide first layers
__host__ __device__ constexpr int cf_nb2(int n1) { return n1 <= 128 ? 2 : 1; }
__host__ __device__ constexpr size_t cf_smem_bytes(int n1, int n2) {
  // ring + A2 + group-1 staging (4 KB per warp) + group-2 staging (nb2 x 4 KB per warp) + align + misc
  return (size_t)kCfStages * cf_stage_bytes(n1, n2) + (size_t)n1 * kTcBM * 2 + 8 * 4096 + 8 * 4096 * cf_nb2(n1) +
         1024 + 1024;
}

struct PipeMaps {
  CUtensorMap a1, a1b, b1, b2;
  CUtensorMap pre1, out1, pre2, out2;
};

template <int N1, int N2, int E1, int E2>
__global__ void __launch_bounds__(kCfThreads, 1)
    gemm_chain_pipe_kernel(const __grid_constant__ PipeMaps cm, EpiParams ep1, EpiParams ep2, int M, int K1,
                           int K1a, int* __restrict__ err) {
  static_assert((N1 == 128 || N1 == 256) && N2 % 32 == 0 && N2 <= 256, "pipelined chain shapes");
  static_assert(E1 == EPI_FWD_SILU || E1 == EPI_HEAD || E1 == EPI_BWD_SILU, "pipelined chain: epilogue 1");
  static_assert(E2 == EPI_FWD_SILU || E2 == EPI_LAST || E2 == EPI_BWD_SILU || E2 == EPI_LINEAR,
                "pipelined chain: epilogue 2");
  constexpr int NH = N1 / kCfJobN;                  // GEMM-1 jobs per tile
  constexpr int NB2 = cf_nb2(N1);
  constexpr uint32_t STAGE = cf_stage_bytes(N1, N2);
  constexpr uint32_t A_BYTES = kTcBM * kTcBK * 2;
  constexpr int NK2 = N1 / kTcBK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;
  uint8_t* sA2 = ring + kCfStages * STAGE;
  uint8_t* sE1 = sA2 + NK2 * A_BYTES;                // group 1: 8 warps x 4 KB
  uint8_t* sE2 = sE1 + 8 * 4096;                     // group 2: 8 warps x NB2 x 4 KB
  uint64_t* full = reinterpret_cast<uint64_t*>(sE2 + 8 * 4096 * NB2);
  uint64_t* empty = full + kCfStages;
  uint64_t* t1full = empty + kCfStages;    // [2]: accumulator slots
  uint64_t* t1empty = t1full + 2;          // [2]
  uint64_t* a2full = t1empty + 2;          // [2]: halves of the on-chip A operand
  uint64_t* a2empty = a2full + 2;          // [2]
  uint64_t* t2full = a2empty + 2;
  uint64_t* t2empty = t2full + 1;
  uint64_t* inb1 = t2empty + 1;            // [8]: group-1 input slots
  uint64_t* inb2 = inb1 + 8;               // [8]: group-2 input slots
  uint64_t* rsbar = inb2 + 8;              // [4]: a quarter's second partial row sum is written
  uint32_t* tslot = reinterpret_cast<uint32_t*>(rsbar + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  float* rowpart = reinterpret_cast<float*>(tslot + 4);   // [4][32]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk1 = (K1 + kTcBK - 1) / kTcBK;
  const int ntiles = (M + kTcBM - 1) / kTcBM;
  const int T = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  auto row0 = [&](int i) { return ((int)blockIdx.x + i * (int)gridDim.x) * kTcBM; };
  // accumulator chunks of 32 columns read with one TMEM load (one wait) in the
  // adjoint-head pairs, two 16-column loads otherwise (measured per pair)
  constexpr bool kLd32 = (E1 == EPI_HEAD);
  constexpr bool kLateG2 = N2 == 256 ? !(E1 == EPI_FWD_SILU && E2 == EPI_FWD_SILU) : (E2 == EPI_LINEAR);

  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < kCfStages; ++s2) {
      mbar_init(&full[s2], 1);
      mbar_init(&empty[s2], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t1full[b], 1);
      mbar_init(&t1empty[b], 8);
      mbar_init(&a2full[b], 8);
      mbar_init(&a2empty[b], 1);
    }
    mbar_init(t2full, 1);
    mbar_init(t2empty, 8);
    for (int q = 0; q < 8; ++q) {
      mbar_init(&inb1[q], 1);
      mbar_init(&inb2[q], 1);
    }
    for (int q = 0; q < 4; ++q) mbar_init(&rsbar[q], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tc_alloc(tslot, 512);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  auto fail = [&]() {
    if (lane == 0) atomicOr(err, kErrTimeout);
    *abort_flag = 1;
  };
  // Row sums of a 32-row quarter split over its two warps (h = 0, 1), combined in
  // that order by warp h = 0.  Warp h = 0 calls this before it releases the
  // accumulator / activation of the tile, so warp h = 1 cannot reach the next
  // tile (and rewrite the slot) before the slot is read.
  auto row_total = [&](int q, int h, int i, float acc, bool& ok) -> float {
    float* part = rowpart + q * 32;
    if (h == 1) {
      part[lane] = acc;
      __syncwarp();
      if (lane == 0) mbar_arrive(&rsbar[q]);
      return 0.0f;
    }
    if (!mbar_wait(&rsbar[q], i & 1)) {
      fail();
      ok = false;
    }
    return acc + part[lane];
  };

  // The MMA job sequence (see above), walked identically by the producer and the MMA thread:
  // g1(i, hf) is GEMM-1 job hf of tile i, g2(i, hf) half hf of tile i's GEMM 2; the walk
  // stops at the first job that returns false (a wait ran out or the kernel is aborting).
  auto walk = [&](auto&& g1, auto&& g2) {
    if (T == 0) return;
    if (!g1(0, 0)) return;
    for (int i = 0; i < T; ++i) {
      if (NH == 1) {
        if (i + 1 < T && !g1(i + 1, 0)) return;
        if (!g2(i, 0)) return;
      } else {
        if (!g1(i, 1)) return;
        if (kLateG2) {
          if (i + 1 < T && !g1(i + 1, 0)) return;
          if (!g2(i, 0)) return;
        } else {
          if (!g2(i, 0)) return;
          if (i + 1 < T && !g1(i + 1, 0)) return;
        }
        if (!g2(i, 1)) return;
      }
    }
  };

  if (warp == 0) {
    // producer
    if (lane == 0) {
      uint32_t g = 0;
      auto slot_free = [&]() -> bool {
        const uint32_t s2 = g % kCfStages, r = g / kCfStages;
        if (g >= (uint32_t)kCfStages && !mbar_wait(&empty[s2], (r - 1) & 1)) {
          fail();
          return false;
        }
        return !*abort_flag;
      };
      auto g1 = [&](int i, int hf) -> bool {
        const int m0 = row0(i);
        for (int kb = 0; kb < nk1; ++kb, ++g) {
          if (!slot_free()) return false;
          const uint32_t s2 = g % kCfStages;
          uint8_t* st = ring + s2 * STAGE;
          mbar_expect_tx(&full[s2], A_BYTES + kCfJobN * kTcBK * 2);
          if (kb * kTcBK < K1a) tma_load_2d(st, &cm.a1, &full[s2], kb * kTcBK, m0);
          else tma_load_2d(st, &cm.a1b, &full[s2], kb * kTcBK - K1a, m0);
          tma_load_2d(st + A_BYTES, &cm.b1, &full[s2], kb * kTcBK, hf * kCfJobN);
        }
        return true;
      };
      auto g2 = [&](int, int hf) -> bool {
        for (int kb = 2 * hf; kb < 2 * hf + 2 && kb < NK2; ++kb, ++g) {
          if (!slot_free()) return false;
          const uint32_t s2 = g % kCfStages;
          mbar_expect_tx(&full[s2], N2 * kTcBK * 2);
          tma_load_2d(ring + s2 * STAGE, &cm.b2, &full[s2], kb * kTcBK, 0);
        }
        return true;
      };
      walk(g1, g2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t id1 = idesc_bf16<kCfJobN>();
      constexpr uint32_t id2 = idesc_bf16<N2>();
      uint32_t g = 0;
      auto g1 = [&](int i, int hf) -> bool {
        const int sj = i * NH + hf, slot = sj & 1, u = sj >> 1;
        if (*abort_flag || !mbar_wait(&t1empty[slot], (u & 1) ^ 1)) { fail(); return false; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(slot * kCfJobN);
        for (int kb = 0; kb < nk1; ++kb, ++g) {
          const uint32_t s2 = g % kCfStages, r = g / kCfStages;
          if (!mbar_wait(&full[s2], r & 1)) { fail(); return false; }
          tc_fence_after();
          const uint32_t a = smem_u32(ring + s2 * STAGE), bb = a + A_BYTES;
#pragma unroll
          for (int k = 0; k < kTcBK / 16; ++k)
            tc_mma(d, sdesc_sw128(a + k * 32), sdesc_sw128(bb + k * 32), id1, (kb > 0 || k > 0) ? 1u : 0u);
          tc_commit(&empty[s2]);
        }
        tc_commit(&t1full[slot]);
        return true;
      };
      auto g2 = [&](int i, int hf) -> bool {
        // half hf of the on-chip A operand (k-blocks 2 hf, 2 hf + 1); the first half also needs acc2 drained
        if (*abort_flag || !mbar_wait(&a2full[hf], i & 1) || (hf == 0 && !mbar_wait(t2empty, (i & 1) ^ 1))) {
          fail();
          return false;
        }
        tc_fence_after();
        for (int kb = 2 * hf; kb < 2 * hf + 2 && kb < NK2; ++kb, ++g) {
          const uint32_t s2 = g % kCfStages, r = g / kCfStages;
          if (!mbar_wait(&full[s2], r & 1)) { fail(); return false; }
          tc_fence_after();
          const uint32_t a = smem_u32(sA2 + kb * A_BYTES), bb = smem_u32(ring + s2 * STAGE);
#pragma unroll
          for (int k = 0; k < kTcBK / 16; ++k)
            tc_mma(tmem + 256, sdesc_sw128(a + k * 32), sdesc_sw128(bb + k * 32), id2, (kb > 0 || k > 0) ? 1u : 0u);
          tc_commit(&empty[s2]);
        }
        tc_commit(&a2empty[hf]);
        if (hf == NH - 1) tc_commit(t2full);
        return true;
      };
      walk(g1, g2);
    }
    __syncwarp();
  } else if (warp < 10) {
    // group 1: acc1 -> epi1 -> A2 (K-major, 128-byte swizzle), plus the HBM side output of the mode
    const int q = warp & 3, ew = warp - 2, h = ew >> 2;
    uint8_t* my = sE1 + ew * 4096;
    uint8_t* islot = my + 2048;                // HEAD / BWD_SILU: the pre-activation chunk
    constexpr bool in1 = (E1 == EPI_HEAD || E1 == EPI_BWD_SILU);
    const bool st_pre = (E1 == EPI_FWD_SILU) && ep1.pre;
    constexpr bool st_out = (E1 == EPI_BWD_SILU);
    uint32_t ipar = 0;
    auto fetch = [&](int i, int c) {
      if (!in1 || i >= T) return;
      if (lane == 0) {
        mbar_expect_tx(&inb1[ew], 2048);
        tma_load_2d(islot, &cm.pre1, &inb1[ew], 32 * c, row0(i) + q * 32);
      }
    };
    if (h < N1 / 32) fetch(0, h);
    int oc = 0;
    bool ok = true;
    for (int i = 0; i < T && ok; ++i) {
      const int mrow = row0(i) + q * 32;
      const int m = mrow + lane;
      const float rs = (m < M && ep1.rowscale) ? ep1.rowscale[m] : 1.0f;
      float2 acc2 = f2_bc(0.0f);
      for (int hf = 0; hf < NH && ok; ++hf) {
      // job (i, hf): accumulator slot sj & 1, columns [128 hf, 128 hf + 128) of the tile
      const int sj = i * NH + hf, slot = sj & 1, u = sj >> 1;
      if (!mbar_wait(&t1full[slot], u & 1) || !mbar_wait(&a2empty[hf], (i & 1) ^ 1)) { fail(); ok = false; break; }
      tc_fence_after();
      if (*abort_flag) { ok = false; break; }
      const uint32_t base = tmem + (uint32_t)(slot * kCfJobN - hf * kCfJobN) + ((uint32_t)(q * 32) << 16);
      for (int c = hf * 4 + h; c < hf * 4 + 4; c += 2) {
        uint32_t zw[16];
        if (in1) {
          if (!mbar_wait(&inb1[ew], ipar)) fail();
          ipar ^= 1u;
          ld_bf16_row_raw(islot, lane, zw);
          // the slot's generic reads are ordered before the next TMA write into it
          fence_async_smem();
          __syncwarp();
          if (c + 2 < N1 / 32) fetch(i, c + 2);
          else fetch(i + 1, h);
        }
        uint8_t* ob = st_pre ? my + (oc & 1) * 2048 : my;
        float v32[kLd32 ? 32 : 1];
        if constexpr (kLd32) tc_ld32(base + (uint32_t)(32 * c), v32);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int nl = 32 * c + 16 * hh;
          float v[16], o2[16];
          if constexpr (kLd32) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = v32[16 * hh + jj];
          } else {
            tc_ld16(base + (uint32_t)nl, v);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            float2 x = make_float2(v[2 * k], v[2 * k + 1]);
            if constexpr (E1 == EPI_FWD_SILU) {
              o2[2 * k] = x.x; o2[2 * k + 1] = x.y;
              x = f2_mul(f2_mul(x, fast_sigmoid2(x)), f2_bc(rs));
            } else {
              const float2 z = bf16_word_pair(zw[8 * hh + k]);
              const float2 sg = fast_sigmoid2(z);
              if constexpr (E1 == EPI_HEAD) {
                // xbar -> the adjoint of the pre-activation of x = u silu(z); row sums of xbar z sigmoid(z)
                acc2 = f2_fma(f2_mul(x, z), sg, acc2);
                x = f2_mul(f2_mul(f2_mul(x, f2_bc(rs)), sg), dsilu_factor2(z, sg));
              } else {
                x = f2_mul(f2_mul(x, sg), dsilu_factor2(z, sg));
              }
            }
            v[2 * k] = x.x; v[2 * k + 1] = x.y;
          }
          uint8_t* kbase = sA2 + (nl / kTcBK) * A_BYTES;
          const int r = q * 32 + lane;
#pragma unroll
          for (int uu = 0; uu < 2; ++uu) {
            const int unit = ((nl % kTcBK) >> 3) + uu;
            uint4 x = make_uint4(pack_bf16x2(v[8 * uu + 0], v[8 * uu + 1]), pack_bf16x2(v[8 * uu + 2], v[8 * uu + 3]),
                                 pack_bf16x2(v[8 * uu + 4], v[8 * uu + 5]), pack_bf16x2(v[8 * uu + 6], v[8 * uu + 7]));
            *reinterpret_cast<uint4*>(kbase + r * 128 + ((unit ^ (r & 7)) << 4)) = x;
          }
          if (st_pre || st_out) {
            if (hh == 0) {
              if (lane == 0) {
                if (st_pre) bulk_wait_read1();
                else bulk_wait_read0();
              }
              __syncwarp();
            }
            st_bf16_half(ob, lane, hh, st_pre ? o2 : v);
          }
        }
        if (st_pre || st_out) {
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(st_pre ? &cm.pre1 : &cm.out1, ob, 32 * c, mrow);
            bulk_commit();
          }
          ++oc;
        }
      }
      if constexpr (E1 == EPI_HEAD) {
        if (hf == NH - 1) {
          const float tot = row_total(q, h, i, acc2.x + acc2.y, ok);
          if (h == 0 && m < M) ep1.ubar[m] += tot;
        }
      }
      tc_fence_before();
      fence_async_smem();          // generic-proxy writes of A2 -> visible to the tensor core
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&t1empty[slot]);
        mbar_arrive(&a2full[hf]);
      }
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  } else {
    // group 2: acc2 -> epi2 -> HBM
    const int q = warp & 3, ew = warp - 10, h = ew >> 2;
    uint8_t* my = sE2 + ew * 4096 * NB2;
    uint8_t* islot = my + 2048;                // BWD_SILU: the pre-activation chunk
    constexpr bool last = E2 == EPI_LAST;
    constexpr bool in2 = E2 == EPI_BWD_SILU;
    const bool pre_out = ep2.pre != nullptr && E2 == EPI_FWD_SILU;
    uint32_t ipar = 0;
    auto fetch = [&](int i, int c) {
      if (!in2 || i >= T) return;
      if (lane == 0) {
        mbar_expect_tx(&inb2[ew], 2048);
        tma_load_2d(islot, &cm.pre2, &inb2[ew], 32 * c, row0(i) + q * 32);
      }
    };
    if (h < N2 / 32) fetch(0, h);
    int oc = 0;
    bool ok = true;
    for (int i = 0; i < T && ok; ++i) {
      const int mrow = row0(i) + q * 32;
      const int m = mrow + lane;
      const float rs = (m < M && ep2.rowscale) ? ep2.rowscale[m] : 1.0f;
      const float srs = (last && m < M) ? ep2.rowsig[m] * rs : 0.0f;
      float2 acc2 = f2_bc(0.0f);
      if (!mbar_wait(t2full, i & 1)) { fail(); break; }
      tc_fence_after();
      if (*abort_flag) break;
      const uint32_t base = tmem + 256u + ((uint32_t)(q * 32) << 16);
      for (int c = h; c < N2 / 32; c += 2) {
        uint32_t zw[16];
        if (in2) {
          if (!mbar_wait(&inb2[ew], ipar)) fail();
          ipar ^= 1u;
          ld_bf16_row_raw(islot, lane, zw);
          fence_async_smem();
          __syncwarp();
          if (c + 2 < N2 / 32) fetch(i, c + 2);
          else fetch(i + 1, h);
        }
        uint8_t* ob = my + (oc % NB2) * 4096;
        float v32[kLd32 ? 32 : 1];
        if constexpr (kLd32) tc_ld32(base + (uint32_t)(32 * c), v32);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float v[16], o2[16];
          if constexpr (kLd32) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = v32[16 * hh + jj];
          } else {
            tc_ld16(base + (uint32_t)(32 * c + 16 * hh), v);
          }
          if constexpr (E2 == EPI_FWD_SILU) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              float2 x = make_float2(v[2 * k], v[2 * k + 1]);
              o2[2 * k] = x.x; o2[2 * k + 1] = x.y;
              x = f2_mul(f2_mul(x, fast_sigmoid2(x)), f2_bc(rs));
              v[2 * k] = x.x; v[2 * k + 1] = x.y;
            }
          } else if constexpr (last) {
            // E_ij = rowscale * sum_n v_n silu(z_n); the pre-activation adjoint
            // sigma_i rowscale v_n silu'(z_n) is the GEMM input of the backward pass
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              const float4 w4 = __ldg(reinterpret_cast<const float4*>(ep2.v + 32 * c + 16 * hh) + k4);
#pragma unroll
              for (int t2 = 0; t2 < 2; ++t2) {
                const int jj = 4 * k4 + 2 * t2;
                const float2 vv = t2 ? make_float2(w4.z, w4.w) : make_float2(w4.x, w4.y);
                const float2 z = make_float2(v[jj], v[jj + 1]);
                const float2 sg = fast_sigmoid2(z);
                acc2 = f2_fma(f2_mul(vv, z), sg, acc2);
                const float2 x = f2_mul(f2_mul(f2_mul(vv, f2_bc(srs)), sg), dsilu_factor2(z, sg));
                v[jj] = x.x; v[jj + 1] = x.y;
              }
            }
          } else if constexpr (in2) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float2 z = bf16_word_pair(zw[8 * hh + k]);
              const float2 sg = fast_sigmoid2(z);
              const float2 x = f2_mul(f2_mul(make_float2(v[2 * k], v[2 * k + 1]), sg), dsilu_factor2(z, sg));
              v[2 * k] = x.x; v[2 * k + 1] = x.y;
            }
          }
          if (hh == 0) {
            if (lane == 0) {
              if (NB2 == 1) bulk_wait_read0();
              else bulk_wait_read1();
            }
            __syncwarp();
          }
          st_bf16_half(ob, lane, hh, v);
          if (pre_out) st_bf16_half(ob + 2048, lane, hh, o2);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&cm.out2, ob, 32 * c, mrow);
          if (pre_out) tma_store_2d(&cm.pre2, ob + 2048, 32 * c, mrow);
          bulk_commit();
        }
        ++oc;
      }
      if constexpr (last) {
        const float tot = row_total(q, h, i, acc2.x + acc2.y, ok);
        if (h == 0 && m < M) {
          ep2.Eout[m] = rs * tot;
          ep2.ubar[m] = ep2.rowsig[m] * tot;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(t2empty);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, 512);
  }
}

// Per-device launch state: a kernel's opt-in to large dynamic shared memory is
// a per-device function attribute, and the SM count sizes the persistent grids.
constexpr int kMaxDevices = 64;
static int g_num_sms[kMaxDevices] = {};

static int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return (d >= 0 && d < kMaxDevices) ? d : 0;
}
static int num_sms(int dev) {
  if (!g_num_sms[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms[dev] = n > 0 ? n : 148;
  }
  return g_num_sms[dev];
}
// opt `kernel` in to `bytes` of dynamic shared memory on device `dev` (once per device)
template <typename K>
static bool smem_opt_in(K kernel, int bytes, bool (&done)[kMaxDevices], int dev, std::string* why) {
  if (done[dev]) return true;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) {
    if (why) *why = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return false;
  }
  done[dev] = true;
  return true;
}

// 2-D tensor map over a row-major [rows][ld] array of `esize`-byte elements,
// box 32 x 32, swizzle matched to the row width of the box.
static bool make_box_map(CUtensorMap* tm, const void* base, int cols, int rows, int ld, int esize) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        esize == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int EPQ>
static bool launch_bn(const GemmArgs& g, const bf16* B, int ldb, cudaStream_t st, int* d_err, std::string* why) {
  static bool attr_set[kMaxDevices] = {};
  const int dev = current_device();
  if (!smem_opt_in(gemm_tc_kernel<BN, EPQ>, kTcSmemMax, attr_set, dev, why)) return false;
  const int nsm = num_sms(dev);
  CUtensorMap ta, ta2, tb;
  const int K1 = g.A2 ? g.K1 : g.K;
  if (!make_tmap(&ta, g.A, (uint64_t)K1, (uint64_t)g.M, (uint64_t)g.lda * 2, kTcBK, kTcBM) ||
      !make_tmap(&ta2, g.A2 ? g.A2 : g.A, (uint64_t)(g.A2 ? g.K - K1 : K1), (uint64_t)g.M,
                 (uint64_t)(g.A2 ? g.lda2 : g.lda) * 2, kTcBK, kTcBM) ||
      !make_tmap(&tb, B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)ldb * 2, kTcBK, BN)) {
    if (why) *why = "cuTensorMapEncodeTiled failed (alignment or extent)";
    return false;
  }
  EpiMaps em;
  memset(&em, 0, sizeof em);
  const bool f32out = (g.epi == EPI_F32);
  bool ok = make_box_map(&em.out, g.out, g.N, g.M, g.ldo, f32out ? 4 : 2);
  if (ok && g.pre) ok = make_box_map(&em.pre, g.pre, g.N, g.M, g.ldp, 2);
  if (ok && g.add) ok = make_box_map(&em.add, g.add, g.N, g.M, g.ld_add, 2);
  if (!ok) {
    if (why) *why = "cuTensorMapEncodeTiled failed for an epilogue operand";
    return false;
  }
  const TcLayout lay = tc_layout<BN, EPQ>(g.epi, g.pre != nullptr);
  if (lay.stages < 2) {
    if (why) *why = "tcgen05 GEMM: shared memory too small for two operand stages";
    return false;
  }
  const size_t smem = tc_smem_bytes<BN, EPQ>(lay);
  const int tiles = ((g.M + kTcBM - 1) / kTcBM) * ((g.N + BN - 1) / BN);
  const int grid = tiles < nsm ? tiles : nsm;
  gemm_tc_kernel<BN, EPQ><<<grid, tc_threads<EPQ>(), smem, st>>>(ta, ta2, tb, em, make_epi(g), lay, g.M, g.N, g.K,
                                                                  K1, d_err);
  return true;
}

bool gemm_tc_bf16(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why) {
  if (g.M <= 0 || g.N <= 0) return true;
  if (!gemm_tc_init(why)) return false;
  const bf16* B = g.Bover ? g.Bover : (g.trans ? g.W->b16T : g.W->b16);
  const int ldb = g.Bover ? g.ldb_over : (g.trans ? g.W->ldT : g.W->ld);
  B += (size_t)g.b_row0 * ldb;
  if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (g.lda % 8) ||
      (ldb % 8) || (g.A2 && ((reinterpret_cast<uintptr_t>(g.A2) & 15) || (g.lda2 % 8) || (g.K1 % kTcBK) ||
                            g.K1 <= 0 || g.K1 >= g.K))) {
    if (why) *why = "tcgen05 GEMM operands must be 16-byte aligned with pitches a multiple of 8 elements";
    return false;
  }
  if (g.add && g.epi != EPI_HEAD) {
    if (why) *why = "the tcgen05 GEMM takes an addend only in the HEAD epilogue (bf16)";
    return false;
  }
  const int tiles = (g.N + 255) / 256;
  if ((g.epi == EPI_HEAD || g.epi == EPI_LAST) && tiles != 1) {
    if (why) *why = "fused head epilogues need N <= 256";
    return false;
  }
  int bn = (g.N + tiles - 1) / tiles;
  bn = (bn + 31) / 32 * 32;
  // four epilogue warps per quarter for the arithmetic epilogues (instantiated
  // for the tile widths the MLP adjoints use), two for plain copies
  const bool wide = (g.epi == EPI_BWD_SILU || g.epi == EPI_LAST) && g.epq != 2;
  switch (bn) {
    case 32: return launch_bn<32, 2>(g, B, ldb, st, d_err, why);
    case 64: return launch_bn<64, 2>(g, B, ldb, st, d_err, why);
    case 96: return launch_bn<96, 2>(g, B, ldb, st, d_err, why);
    case 128:
      return wide ? launch_bn<128, 4>(g, B, ldb, st, d_err, why) : launch_bn<128, 2>(g, B, ldb, st, d_err, why);
    case 160: return launch_bn<160, 2>(g, B, ldb, st, d_err, why);
    case 192: return launch_bn<192, 2>(g, B, ldb, st, d_err, why);
    case 224: return launch_bn<224, 2>(g, B, ldb, st, d_err, why);
    default:
      return wide ? launch_bn<256, 4>(g, B, ldb, st, d_err, why) : launch_bn<256, 2>(g, B, ldb, st, d_err, why);
  }
}


template <int N1, int N2, int E1, int E2>
static bool launch_chain_pipe(const GemmArgs& g1, const GemmArgs& g2, const bf16* B1, int ldb1, const bf16* B2,
                              int ldb2, cudaStream_t st, int* d_err, std::string* why) {
  constexpr size_t smem = cf_smem_bytes(N1, N2);
  static_assert(smem <= 232448, "pipelined chain shared memory");
  static bool attr_set[kMaxDevices] = {};
  const int dev = current_device();
  if (!smem_opt_in(gemm_chain_pipe_kernel<N1, N2, E1, E2>, (int)smem, attr_set, dev, why)) return false;
  const int nsm = num_sms(dev);
  const int K1a = g1.A2 ? g1.K1 : g1.K;
  PipeMaps cm;
  memset(&cm, 0, sizeof cm);
  bool ok = make_tmap(&cm.a1, g1.A, (uint64_t)K1a, (uint64_t)g1.M, (uint64_t)g1.lda * 2, kTcBK, kTcBM) &&
            make_tmap(&cm.a1b, g1.A2 ? g1.A2 : g1.A, (uint64_t)(g1.A2 ? g1.K - K1a : K1a), (uint64_t)g1.M,
                      (uint64_t)(g1.A2 ? g1.lda2 : g1.lda) * 2, kTcBK, kTcBM) &&
            make_tmap(&cm.b1, B1, (uint64_t)g1.K, (uint64_t)g1.N, (uint64_t)ldb1 * 2, kTcBK, kCfJobN) &&
            make_tmap(&cm.b2, B2, (uint64_t)g2.K, (uint64_t)g2.N, (uint64_t)ldb2 * 2, kTcBK, N2);
  if (ok && g1.pre) ok = make_box_map(&cm.pre1, g1.pre, g1.N, g1.M, g1.ldp, 2);
  if (ok && g1.epi == EPI_BWD_SILU) ok = make_box_map(&cm.out1, g1.out, g1.N, g1.M, g1.ldo, 2);
  if (ok && g2.pre && (g2.epi == EPI_FWD_SILU || g2.epi == EPI_BWD_SILU))
    ok = make_box_map(&cm.pre2, g2.pre, g2.N, g2.M, g2.ldp, 2);
  if (ok) ok = make_box_map(&cm.out2, g2.out, g2.N, g2.M, g2.ldo, 2);
  if (!ok) {
    if (why) *why = "cuTensorMapEncodeTiled failed (chain)";
    return false;
  }
  const int tiles = (g1.M + kTcBM - 1) / kTcBM;
  const int grid = tiles < nsm ? tiles : nsm;
  gemm_chain_pipe_kernel<N1, N2, E1, E2><<<grid, kCfThreads, smem, st>>>(cm, make_epi(g1), make_epi(g2), g1.M,
                                                                          g1.K, K1a, d_err);
  return true;
}

// Two consecutive layers in one kernel (see gemm_chain_pipe_kernel) for the
// pairs it is instantiated for.  Returns false with `why` empty when the pair
// is not supported (the caller then runs the two GEMMs separately).
bool gemm_chain_bf16(const GemmArgs& g1, const GemmArgs& g2, cudaStream_t st, int* d_err, std::string* why) {
  if (why) why->clear();
  if (g1.M <= 0) return true;
  if (g2.K != g1.N || g2.M != g1.M || g2.A2 || g1.add || g2.add) return false;
  if (!gemm_tc_init(why)) return false;
  const bf16* B1 = g1.Bover ? g1.Bover : (g1.trans ? g1.W->b16T : g1.W->b16);
  const int ldb1 = g1.Bover ? g1.ldb_over : (g1.trans ? g1.W->ldT : g1.W->ld);
  B1 += (size_t)g1.b_row0 * ldb1;
  const bf16* B2 = g2.Bover ? g2.Bover : (g2.trans ? g2.W->b16T : g2.W->b16);
  const int ldb2 = g2.Bover ? g2.ldb_over : (g2.trans ? g2.W->ldT : g2.W->ld);
  B2 += (size_t)g2.b_row0 * ldb2;
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (!al(g1.A) || !al(B1) || !al(B2) || (g1.lda % 8) || (ldb1 % 8) || (ldb2 % 8)) return false;
  if (g1.A2 && (!al(g1.A2) || (g1.lda2 % 8) || (g1.K1 % kTcBK) || g1.K1 <= 0 || g1.K1 >= g1.K)) return false;
  // the pipelined kernel
  const bool e1ok = g1.epi == EPI_FWD_SILU || (g1.epi == EPI_HEAD && g1.pre && g1.ubar) ||
                    (g1.epi == EPI_BWD_SILU && g1.pre && g1.out);
  const bool last_ok = g2.epi == EPI_LAST && g2.v && g2.rowsig && g2.Eout && g2.ubar && al(g2.v) &&
                       g1.epi != EPI_HEAD;
  const bool e2ok = g2.epi == EPI_FWD_SILU || last_ok || (g2.epi == EPI_BWD_SILU && g2.pre) || g2.epi == EPI_LINEAR;
  if (e1ok && e2ok) {
    // instantiated for the pairs of the MLPs' forward and adjoint passes
#define PIPE(n1, n2, e1, e2) \
  if (g1.N == n1 && g2.N == n2 && g1.epi == e1 && g2.epi == e2) \
    return launch_chain_pipe<n1, n2, e1, e2>(g1, g2, B1, ldb1, B2, ldb2, st, d_err, why);
    PIPE(128, 256, EPI_FWD_SILU, EPI_FWD_SILU)
    PIPE(256, 256, EPI_FWD_SILU, EPI_FWD_SILU)
    PIPE(256, 256, EPI_FWD_SILU, EPI_LAST)
    PIPE(256, 256, EPI_HEAD, EPI_BWD_SILU)
    PIPE(256, 128, EPI_HEAD, EPI_BWD_SILU)
    PIPE(256, 64, EPI_BWD_SILU, EPI_LINEAR)
#undef PIPE
  }
  return false;
}


// ---------------------------------------------------------------------------
// TF32 GEMM on tcgen05 (kind::tf32) for the float32-storage precisions:
//   C[M x N] = A[M x K] B^T, A float32 activations [M][lda], B float32 weights
//   [N][ldb] (K contiguous), float32 accumulation in TMEM, with the float32
//   path's epilogues (SiLU forward with the pre-activation store and the
//   per-row scale, float32 output with an addend, SiLU adjoint, linear).
// The tensor core reads each float32 operand as TF32 (10-bit mantissa): the
// paper's production setting (Table IV: float64 final, float32 weights and
// activations, TF32 matrix multiplications).
// Persistent: CTA b walks 128 x BN tiles; warp 0 issues TMA loads of 128 x 32
// (A) and BN x 32 (B) float32 tiles (128-byte rows, 128-byte swizzle) into a
// shared-memory ring, warp 1 owns two BN-column TMEM accumulators and issues
// tcgen05.mma.kind::tf32 (K = 8 per instruction) from one thread, 8 epilogue
// warps (2 per TMEM lane quarter, alternating 32-column chunks) read the
// accumulator with tcgen05.ld and write their rows with 16-byte stores.
// ---------------------------------------------------------------------------
constexpr int kT32BK = 32;                     // float32 elements per 128-byte operand row
constexpr int kT32Threads = 64 + 8 * 32;

template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_tf32() {
  // D f32, A tf32, B tf32, both K-major, M = 128, N = BN
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

template <int BN>
__host__ __device__ constexpr int t32_stage_bytes() {
  return 128 * kT32BK * 4 + BN * kT32BK * 4;
}
template <int BN>
__host__ __device__ constexpr int t32_stages() {
  return (kTcSmemMax - 1024 - 1024) / t32_stage_bytes<BN>() > 6 ? 6
                                                               : (kTcSmemMax - 1024 - 1024) / t32_stage_bytes<BN>();
}
template <int BN>
__host__ __device__ constexpr int t32_smem_bytes() {
  return t32_stages<BN>() * t32_stage_bytes<BN>() + 1024 + 1024;
}

// 32 consecutive float32 columns of one row: epilogue of the float32 path
__device__ __forceinline__ void t32_epilogue(const EpiParams& ep, int m, int n, int N, float (&v)[32]) {
  const bool full = (n + 32 <= N) && ep.vec;
  if (ep.epi == EPI_FWD_SILU) {
    const float rs = ep.rowscale ? ep.rowscale[m] : 1.0f;
    if (ep.pre) {
      float* pp = reinterpret_cast<float*>(ep.pre) + (size_t)m * ep.ldp + n;
      if (full) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          reinterpret_cast<float4*>(pp)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (n + j < N) pp[j] = v[j];
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = v[j] * epi_sigmoid(v[j]) * rs;
  } else if (ep.epi == EPI_F32) {
    if (ep.add) {
      const float* a = reinterpret_cast<const float*>(ep.add) + (size_t)m * ep.ld_add + n;
      if (full) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 x = reinterpret_cast<const float4*>(a)[k];
          v[4 * k] += x.x; v[4 * k + 1] += x.y; v[4 * k + 2] += x.z; v[4 * k + 3] += x.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (n + j < N) v[j] += a[j];
      }
    }
  } else if (ep.epi == EPI_BWD_SILU) {
    const float* zp = reinterpret_cast<const float*>(ep.pre) + (size_t)m * ep.ldp + n;
    float z[32];
    if (full) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 x = reinterpret_cast<const float4*>(zp)[k];
        z[4 * k] = x.x; z[4 * k + 1] = x.y; z[4 * k + 2] = x.z; z[4 * k + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = (n + j < N) ? zp[j] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float sg = epi_sigmoid(z[j]);
      v[j] = v[j] * sg * (1.0f + z[j] * (1.0f - sg));
    }
  }
  float* o = reinterpret_cast<float*>(ep.out) + (size_t)m * ep.ldo + n;
  if (full) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      reinterpret_cast<float4*>(o)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (n + j < N) o[j] = v[j];
  }
}

template <int BN>
__global__ void __launch_bounds__(kT32Threads, 1)
    gemm_tf32_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiParams ep,
                     int M, int N, int K, int* __restrict__ err) {
  constexpr int STAGES = t32_stages<BN>();
  constexpr uint32_t A_BYTES = 128 * kT32BK * 4;
  constexpr uint32_t B_BYTES = BN * kT32BK * 4;
  constexpr uint32_t COLS = tc_tmem_cols<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;   // [2]
  uint64_t* tempty = tfull + 2;       // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (K + kT32BK - 1) / kT32BK;
  const int tiles_m = (M + 127) / 128, tiles_n = (N + BN - 1) / BN;
  const int ntiles = tiles_m * tiles_n;
  auto tm0 = [&](int tt) { return (tt / tiles_n) * 128; };
  auto tn0 = [&](int tt) { return (tt % tiles_n) * BN; };

  if (threadIdx.x == 0) {
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
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
      uint32_t g = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        const int m0 = tm0(t), n0 = tn0(t);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const uint32_t q = g % STAGES, r = g / STAGES;
          if (g >= (uint32_t)STAGES && !mbar_wait(&empty[q], (r - 1) & 1)) {
            atomicOr(err, kErrTimeout);
            *abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full[q], A_BYTES + B_BYTES);
          tma_load_2d(sA + q * A_BYTES, &tmA, &full[q], kb * kT32BK, m0);
          tma_load_2d(sB + q * B_BYTES, &tmB, &full[q], kb * kT32BK, n0);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32<BN>();
      uint32_t g = 0;
      int lt = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
        const int b = lt & 1, use = lt >> 1;
        bool ok = !*abort_flag && mbar_wait(&tempty[b], (use & 1) ^ 1);
        if (ok) {
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * COLS);
          for (int kb = 0; kb < nk; ++kb, ++g) {
            const uint32_t q = g % STAGES, r = g / STAGES;
            if (!mbar_wait(&full[q], r & 1)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sA + q * A_BYTES), b_addr = smem_u32(sB + q * B_BYTES);
#pragma unroll
            for (int k = 0; k < kT32BK / 8; ++k)   // 8 tf32 = 32 bytes per instruction
              tc_mma_tf32(dt, sdesc_sw128(a_addr + k * 32), sdesc_sw128(b_addr + k * 32), idesc,
                          (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[q]);
          }
        }
        if (!ok) {
          atomicOr(err, kErrTimeout);
          *abort_flag = 1;
        }
        tc_commit(&tfull[b]);
        if (!ok) break;
      }
    }
    __syncwarp();
  } else {
    const int q = warp & 3;        // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2; // 0 or 1: alternating 32-column chunks
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int b = lt & 1, use = lt >> 1;
      if (!mbar_wait(&tfull[b], use & 1)) {
        if (lane == 0) atomicOr(err, kErrTimeout);
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
        if (m < M) t32_epilogue(ep, m, n0 + 32 * c, N, v);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, 2 * COLS);
  }
}

static bool make_tmap_f32(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                          uint32_t box_inner, uint32_t box_outer) {
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        inner * 4 < row_bytes ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN>
static bool launch_tf32(const GemmArgs& g, const float* B, int ldb, cudaStream_t st, int* d_err, std::string* why) {
  static bool attr_set[kMaxDevices] = {};
  const int dev = current_device();
  constexpr int smem = t32_smem_bytes<BN>();
  static_assert(smem <= kTcSmemMax, "tf32 GEMM shared memory");
  if (!smem_opt_in(gemm_tf32_kernel<BN>, smem, attr_set, dev, why)) return false;
  CUtensorMap ta, tb;
  if (!make_tmap_f32(&ta, g.A, (uint64_t)g.K, (uint64_t)g.M, (uint64_t)g.lda * 4, kT32BK, 128) ||
      !make_tmap_f32(&tb, B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)ldb * 4, kT32BK, BN)) {
    if (why) *why = "cuTensorMapEncodeTiled failed (tf32 operands)";
    return false;
  }
  const int tiles = ((g.M + 127) / 128) * ((g.N + BN - 1) / BN);
  const int nsm = num_sms(dev);
  const int grid = tiles < nsm ? tiles : nsm;
  gemm_tf32_kernel<BN><<<grid, kT32Threads, smem, st>>>(ta, tb, make_epi(g), g.M, g.N, g.K, d_err);
  return true;
}

bool gemm_tc_tf32(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why) {
  if (g.M <= 0 || g.N <= 0) return true;
  if (!gemm_tc_init(why)) return false;
  if (g.A2 || g.Bover || g.b_row0 || !(g.epi == EPI_FWD_SILU || g.epi == EPI_F32 || g.epi == EPI_BWD_SILU ||
                                       g.epi == EPI_LINEAR)) {
    if (why) *why = "tf32 GEMM: unsupported operand form or epilogue";
    return false;
  }
  const float* B = g.trans ? g.W->f32T : g.W->f32;
  const int ldb = g.trans ? g.W->ldT : g.W->ld;
  if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (g.lda % 4) ||
      (ldb % 4)) {
    if (why) *why = "tf32 GEMM operands must be 16-byte aligned with pitches a multiple of 4 elements";
    return false;
  }
  const int tiles = (g.N + 255) / 256;
  int bn = (g.N + tiles - 1) / tiles;
  bn = (bn + 31) / 32 * 32;
  switch (bn) {
    case 32: return launch_tf32<32>(g, B, ldb, st, d_err, why);
    case 64: return launch_tf32<64>(g, B, ldb, st, d_err, why);
    case 96: return launch_tf32<96>(g, B, ldb, st, d_err, why);
    case 128: return launch_tf32<128>(g, B, ldb, st, d_err, why);
    case 160: return launch_tf32<160>(g, B, ldb, st, d_err, why);
    case 192: return launch_tf32<192>(g, B, ldb, st, d_err, why);
    case 224: return launch_tf32<224>(g, B, ldb, st, d_err, why);
    default: return launch_tf32<256>(g, B, ldb, st, d_err, why);
  }
}

}  // namespace alg
