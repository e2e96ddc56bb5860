// allegro_neighbors_noalloc: the all-pairs neighbour search of one small
// structure without any device allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example an MD engine whose device memory is owned by its own pool
// allocator (allocating behind its back fragments or exhausts that pool),
// code that runs between cudaStreamBeginCapture and EndCapture (where
// cudaMalloc is not allowed), or a long steady-state loop that has to keep a
// fixed memory footprint.  Such callers cannot create a context, whose arena
// is allocated on demand.
//
// Scratch (per-atom counts, row offsets and the edge total) lives in one
// file-scope __device__ array of fixed size (kScratchInts ints, 128 KiB).  Every GPU that
// loads this library holds that array until the process exits.  The first
// call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture.  All calls on a device share the
// array and it keeps the previous call's contents: every entry a call reads is
// written earlier in the same call (counts, offsets, total), so nothing needs
// clearing, and calls that overlap on the GPU (different streams, or host
// threads racing) corrupt each other's results.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/allegro.h"

namespace {

constexpr int kNoAllocMaxAtoms = 16384;
// [0, kMax]: per-atom counts; [kMax+1, 2 kMax+2): row offsets (n+1 entries);
// then the edge total.
constexpr int kScratchInts = 2 * (kNoAllocMaxAtoms + 1) + 8;

static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

struct NoAllocCell {
  double cell[9];
  int pbc[3];
  int nimg[3];
};

__device__ __forceinline__ bool noalloc_pair(const double* __restrict__ pi, const double* __restrict__ pj,
                                             const double* cell, int S0, int S1, int S2, double rc2) {
  double s0 = (double)S0, s1 = (double)S1, s2 = (double)S2, d[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    double off = __dadd_rn(__dadd_rn(__dmul_rn(s0, cell[x]), __dmul_rn(s1, cell[3 + x])), __dmul_rn(s2, cell[6 + x]));
    d[x] = __dsub_rn(__dadd_rn(pj[x], off), pi[x]);
  }
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < rc2;
}

// fill == false: count[i] = number of edges of centre i.
// fill == true: write edges of centre i at row[i] (rows ascending in i).
__global__ void noalloc_search_kernel(bool fill, const double* __restrict__ pos, int n, NoAllocCell c, double rc2,
                                      int* __restrict__ scratch, int64_t cap, int32_t* __restrict__ oi,
                                      int32_t* __restrict__ oj, int32_t* __restrict__ oS) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int* count = scratch;
  const int* row = scratch + (kNoAllocMaxAtoms + 1);
  const double pi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  int k = 0;
  const long long base = fill ? row[i] : 0;
  for (int j = 0; j < n; ++j)
    for (int S0 = -c.nimg[0]; S0 <= c.nimg[0]; ++S0)
      for (int S1 = -c.nimg[1]; S1 <= c.nimg[1]; ++S1)
        for (int S2 = -c.nimg[2]; S2 <= c.nimg[2]; ++S2) {
          if (j == i && S0 == 0 && S1 == 0 && S2 == 0) continue;
          if (!noalloc_pair(pi, pos + 3 * j, c.cell, S0, S1, S2, rc2)) continue;
          if (fill) {
            const long long o = base + k;
            if (o < cap) {
              oi[o] = i;
              oj[o] = j;
              oS[3 * o] = S0; oS[3 * o + 1] = S1; oS[3 * o + 2] = S2;
            }
          }
          ++k;
        }
  if (!fill) count[i] = k;
}

// One block: exclusive scan of count[0..n) into row[0..n]; row[n] = total.
__global__ void noalloc_scan_kernel(int n, int* __restrict__ scratch) {
  const int* count = scratch;
  int* row = scratch + (kNoAllocMaxAtoms + 1);
  int* total = scratch + 2 * (kNoAllocMaxAtoms + 1) + 1;
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = t * per, e = min(n, b + per);
  int s = 0;
  for (int q = b; q < e; ++q) s += count[q];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v = (t >= o) ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int q = b; q < e; ++q) {
    row[q] = run;
    run += count[q];
  }
  if (t == 1023) {
    row[n] = part[1023];
    *total = part[1023];
  }
}

std::mutex g_mu;
int* g_dev_ptr[64] = {nullptr};

}  // namespace

extern "C" allegro_status allegro_neighbors_noalloc(const double* pos, int64_t n_atoms, const double* cell,
                                                    const uint8_t* pbc, double r_c, int32_t* i, int32_t* j,
                                                    int32_t* shift, int64_t cap, int64_t* n_edges,
                                                    void* stream) {
  if (n_atoms < 0 || n_atoms > kNoAllocMaxAtoms) {
    fprintf(stderr, "allegro_neighbors_noalloc: n_atoms = %lld exceeds the fixed scratch limit of %d atoms\n",
            (long long)n_atoms, kNoAllocMaxAtoms);
    return ALLEGRO_E_CAPACITY;
  }
  if (!n_edges || !(r_c > 0) || cap < 0 || (n_atoms > 0 && !pos) || (cap > 0 && (!i || !j || !shift)))
    return ALLEGRO_E_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ALLEGRO_E_CUDA;
  int* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return ALLEGRO_E_CUDA;
      }
      g_dev_ptr[dev] = static_cast<int*>(p);
    }
    scratch = g_dev_ptr[dev];
  }
  NoAllocCell c;
  memset(&c, 0, sizeof c);
  for (int k = 0; k < 3; ++k) c.pbc[k] = (cell && (!pbc || pbc[k])) ? 1 : 0;
  if (cell) {
    memcpy(c.cell, cell, sizeof c.cell);
    const double* a = c.cell;
    const double* b = c.cell + 3;
    const double* cc = c.cell + 6;
    double bc[3] = {b[1] * cc[2] - b[2] * cc[1], b[2] * cc[0] - b[0] * cc[2], b[0] * cc[1] - b[1] * cc[0]};
    double ca[3] = {cc[1] * a[2] - cc[2] * a[1], cc[2] * a[0] - cc[0] * a[2], cc[0] * a[1] - cc[1] * a[0]};
    double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double vol = fabs(a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]);
    const double* cr[3] = {bc, ca, ab};
    for (int k = 0; k < 3; ++k) {
      double w = vol / sqrt(cr[k][0] * cr[k][0] + cr[k][1] * cr[k][1] + cr[k][2] * cr[k][2]);
      if (!(w > 0) || !std::isfinite(w)) return ALLEGRO_E_INVALID;
      // positions within fractional coordinates [-0.5, 1.5): spread < 2 cell widths
      c.nimg[k] = c.pbc[k] ? (int)ceil(r_c / w) + 2 : 0;
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)n_atoms;
  const double rc2 = r_c * r_c;
  const int blocks = (n + 127) / 128;
  if (n > 0) noalloc_search_kernel<<<blocks, 128, 0, st>>>(false, pos, n, c, rc2, scratch, 0, nullptr, nullptr, nullptr);
  noalloc_scan_kernel<<<1, 1024, 0, st>>>(n, scratch);
  if (cudaGetLastError() != cudaSuccess) return ALLEGRO_E_CUDA;
  int total = 0;
  if (cudaMemcpyAsync(&total, scratch + 2 * (kNoAllocMaxAtoms + 1) + 1, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ALLEGRO_E_CUDA;
  *n_edges = total;
  if (total > cap) return ALLEGRO_E_CAPACITY;
  if (n > 0) noalloc_search_kernel<<<blocks, 128, 0, st>>>(true, pos, n, c, rc2, scratch, cap, i, j, shift);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return ALLEGRO_E_CUDA;
  return ALLEGRO_OK;
}
