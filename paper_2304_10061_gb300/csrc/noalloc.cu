// allegro_neighbors_noalloc: the all-pairs neighbour search of one small
// structure without any device allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example an MD engine whose device memory is owned by its own pool
// allocator (allocating behind its back fragments or exhausts that pool), or a
// long steady-state loop that has to keep a fixed memory footprint.  Such
// callers cannot create a context, whose arena is allocated on demand.
//
// Scratch (per-atom counts, row offsets, the edge total and a flag word) lives
// in one file-scope __device__ array of fixed size (kScratchInts ints, about
// 128 KiB).  Every GPU that loads this library holds that array until the
// process exits.  The first call on a device looks up the array's device
// address with cudaGetSymbolAddress (once per device, with that device
// current); make that first call before any stream capture.  All calls on a
// device share the array and it keeps the previous call's contents: the flag
// word is cleared at the start of each call and every other entry a call reads
// is written earlier in the same call (counts, offsets, total).  Calls that
// overlap on the GPU (different streams, or host threads racing) corrupt each
// other's results.  Each call synchronises its stream: it reads the edge count
// back to the host before the fill pass.
//
// Candidate images are chosen per pair: with f = frac(pos_j - pos_i) along a
// periodic axis k, |d| >= w_k |f_k + S_k| (w_k the perpendicular width), so
// only S_k in (-f_k - r_c/w_k, -f_k + r_c/w_k) can hold an edge.  The window
// is widened by a relative 1e-9 plus a bound on the float64 rounding of the
// displacement (a few ulps of the magnitudes it adds, over w_k), and every
// candidate takes the exact float64 test, so positions need not be wrapped
// into the cell.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>

#include "../../include/allegro.h"

namespace {

constexpr int kNoAllocMaxAtoms = 16384;
// largest cutoff-to-width ratio along a periodic axis (image reach per side)
constexpr double kMaxReach = 4.0;
// largest number of (pair, image) candidates a call may test
constexpr double kMaxCandidates = 6.0e10;
// [0, kMax]: per-atom counts; [kMax+1, 2 kMax+2): row offsets (n+1 entries);
// then (8-byte aligned) the edge total as int64 and the flag word.
constexpr int kRowBase = kNoAllocMaxAtoms + 1;
constexpr int kTailBase = 2 * (kNoAllocMaxAtoms + 1);   // even: 8-byte aligned
constexpr int kScratchInts = kTailBase + 8;
constexpr int kFlagBadPos = 1;

static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

struct NoAllocCell {
  double cell[9];
  double inv[9];     // frac = d inv (row vector times matrix)
  double reach[3];   // r_c / w_k on periodic axes, 0 otherwise
  double invw[3];    // 1 / w_k
  double cmax;       // largest |component| of the cell
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

// fill == false: count[i] = number of edges of centre i; non-finite positions
// set the flag word.  fill == true: write edges of centre i at row[i] (rows
// ascending in i).
__global__ void noalloc_search_kernel(bool fill, const double* __restrict__ pos, int n, NoAllocCell c, double rc2,
                                      int* __restrict__ scratch, int64_t cap, int32_t* __restrict__ oi,
                                      int32_t* __restrict__ oj, int32_t* __restrict__ oS) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int* count = scratch;
  const int* row = scratch + kRowBase;
  int* flags = scratch + kTailBase + 2;
  const double pi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  if (!(isfinite(pi[0]) && isfinite(pi[1]) && isfinite(pi[2]))) {
    if (!fill) {
      atomicOr(flags, kFlagBadPos);
      count[i] = 0;
    }
    return;
  }
  int k = 0;
  const long long base = fill ? row[i] : 0;
  for (int j = 0; j < n; ++j) {
    const double* pj = pos + 3 * j;
    const double dx = pj[0] - pi[0], dy = pj[1] - pi[1], dz = pj[2] - pi[2];
    if (!(isfinite(dx) && isfinite(dy) && isfinite(dz))) continue;   // j's own thread flags it
    // bound on the rounding of the exact test's displacement (a few ulps of the
    // largest magnitude it adds), as a fraction of the width along each axis
    const double mag = fmax(fmax(fabs(pi[0]), fabs(pi[1])), fabs(pi[2])) +
                       fmax(fmax(fabs(pj[0]), fabs(pj[1])), fabs(pj[2]));
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (c.reach[a] > 0.0) {
        const double f = dx * c.inv[a] + dy * c.inv[3 + a] + dz * c.inv[6 + a];
        if (!(fabs(f) < 1e8)) {   // pairs this far apart (in cells) are rejected as bad input
          if (!fill) atomicOr(flags, kFlagBadPos);
          lo[a] = 1; hi[a] = 0;
          continue;
        }
        const double win = c.reach[a] * (1.0 + 1e-9) +
                           4e-15 * (mag + (fabs(f) + c.reach[a] + 1.0) * c.cmax) * c.invw[a];
        lo[a] = (int)ceil(-f - win);
        hi[a] = (int)floor(-f + win);
      } else {
        lo[a] = hi[a] = 0;
      }
    }
    for (int S0 = lo[0]; S0 <= hi[0]; ++S0)
      for (int S1 = lo[1]; S1 <= hi[1]; ++S1)
        for (int S2 = lo[2]; S2 <= hi[2]; ++S2) {
          if (j == i && S0 == 0 && S1 == 0 && S2 == 0) continue;
          if (!noalloc_pair(pi, pj, c.cell, S0, S1, S2, rc2)) continue;
          if (fill) {
            const long long o = base + k;
            if (o >= 0 && o < cap) {
              oi[o] = i;
              oj[o] = j;
              oS[3 * o] = S0; oS[3 * o + 1] = S1; oS[3 * o + 2] = S2;
            }
          }
          ++k;
        }
  }
  if (!fill) count[i] = k;
}

// One block: exclusive scan of count[0..n) into row[0..n] (int64 running sums,
// stored as int32; the host rejects totals beyond INT32_MAX before the fill
// pass reads them); the total as int64.
__global__ void noalloc_scan_kernel(int n, int* __restrict__ scratch) {
  const int* count = scratch;
  int* row = scratch + kRowBase;
  long long* total = reinterpret_cast<long long*>(scratch + kTailBase);
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = t * per, e = min(n, b + per);
  long long s = 0;
  for (int q = b; q < e; ++q) s += count[q];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long v = (t >= o) ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = part[t] - s;
  for (int q = b; q < e; ++q) {
    row[q] = (int)run;
    run += count[q];
  }
  if (t == 1023) {
    row[n] = (int)part[1023];
    *total = part[1023];
  }
}

std::mutex g_mu;
int* g_dev_ptr[64] = {nullptr};

bool invert3(const double* m, double* inv) {
  const double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                     m[2] * (m[3] * m[7] - m[4] * m[6]);
  if (!(fabs(det) > 0) || !std::isfinite(det)) return false;
  const double id = 1.0 / det;
  inv[0] = (m[4] * m[8] - m[5] * m[7]) * id;
  inv[1] = (m[2] * m[7] - m[1] * m[8]) * id;
  inv[2] = (m[1] * m[5] - m[2] * m[4]) * id;
  inv[3] = (m[5] * m[6] - m[3] * m[8]) * id;
  inv[4] = (m[0] * m[8] - m[2] * m[6]) * id;
  inv[5] = (m[2] * m[3] - m[0] * m[5]) * id;
  inv[6] = (m[3] * m[7] - m[4] * m[6]) * id;
  inv[7] = (m[1] * m[6] - m[0] * m[7]) * id;
  inv[8] = (m[0] * m[4] - m[1] * m[3]) * id;
  return true;
}

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
  if (!n_edges || !(r_c > 0) || !std::isfinite(r_c) || cap < 0 || (n_atoms > 0 && !pos) ||
      (cap > 0 && (!i || !j || !shift)))
    return ALLEGRO_E_INVALID;
  NoAllocCell c;
  memset(&c, 0, sizeof c);
  double images = 1.0;
  if (cell) {
    memcpy(c.cell, cell, sizeof c.cell);
    for (double v : c.cell)
      if (!std::isfinite(v)) return ALLEGRO_E_INVALID;
    if (!invert3(c.cell, c.inv)) return ALLEGRO_E_INVALID;
    for (double v : c.cell) c.cmax = std::max(c.cmax, fabs(v));
    const double* a = c.cell;
    const double* b = c.cell + 3;
    const double* cc = c.cell + 6;
    const double bc[3] = {b[1] * cc[2] - b[2] * cc[1], b[2] * cc[0] - b[0] * cc[2], b[0] * cc[1] - b[1] * cc[0]};
    const double ca[3] = {cc[1] * a[2] - cc[2] * a[1], cc[2] * a[0] - cc[0] * a[2], cc[0] * a[1] - cc[1] * a[0]};
    const double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double vol = fabs(a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]);
    const double* cr[3] = {bc, ca, ab};
    for (int k = 0; k < 3; ++k) {
      if (pbc && !pbc[k]) continue;
      const double w = vol / sqrt(cr[k][0] * cr[k][0] + cr[k][1] * cr[k][1] + cr[k][2] * cr[k][2]);
      if (!(w > 0) || !std::isfinite(w)) return ALLEGRO_E_INVALID;
      const double reach = r_c / w;
      if (reach > kMaxReach) {
        fprintf(stderr, "allegro_neighbors_noalloc: r_c / cell width = %g along axis %d exceeds %g\n", reach, k,
                kMaxReach);
        return ALLEGRO_E_INVALID;
      }
      c.reach[k] = reach;
      c.invw[k] = 1.0 / w;
      images *= 2.0 * ceil(reach * (1.0 + 1e-6)) + 1.0;
    }
  }
  if ((double)n_atoms * (double)n_atoms * images > kMaxCandidates) {
    fprintf(stderr, "allegro_neighbors_noalloc: %g candidate (pair, image) tests exceed the limit of %g\n",
            (double)n_atoms * (double)n_atoms * images, kMaxCandidates);
    return ALLEGRO_E_CAPACITY;
  }
  if (n_atoms == 0) {
    *n_edges = 0;
    return ALLEGRO_OK;
  }
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
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)n_atoms;
  const double rc2 = r_c * r_c;
  const int blocks = (n + 127) / 128;
  if (cudaMemsetAsync(scratch + kTailBase + 2, 0, sizeof(int), st) != cudaSuccess) return ALLEGRO_E_CUDA;
  noalloc_search_kernel<<<blocks, 128, 0, st>>>(false, pos, n, c, rc2, scratch, 0, nullptr, nullptr, nullptr);
  noalloc_scan_kernel<<<1, 1024, 0, st>>>(n, scratch);
  if (cudaGetLastError() != cudaSuccess) return ALLEGRO_E_CUDA;
  int tail[4] = {0, 0, 0, 0};   // int64 total, flag word, unused
  if (cudaMemcpyAsync(tail, scratch + kTailBase, sizeof tail, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ALLEGRO_E_CUDA;
  long long total = 0;
  memcpy(&total, tail, sizeof total);
  if (tail[2] & kFlagBadPos) {
    fprintf(stderr, "allegro_neighbors_noalloc: a position is not finite or lies 1e8 cells from another\n");
    return ALLEGRO_E_INVALID;
  }
  *n_edges = total;
  if (total > cap || total > (long long)INT32_MAX) return ALLEGRO_E_CAPACITY;
  noalloc_search_kernel<<<blocks, 128, 0, st>>>(true, pos, n, c, rc2, scratch, cap, i, j, shift);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return ALLEGRO_E_CUDA;
  return ALLEGRO_OK;
}
