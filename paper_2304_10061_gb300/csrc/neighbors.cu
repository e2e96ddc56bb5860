// Ordered neighbour pairs within r_c (Sec. "Allegro": E_i = sum_j E_ij over
// ordered pairs; Sec. "Species-dependent cutoffs").
//
// Cell list: atoms are binned by fractional coordinate into cells whose
// perpendicular widths are at least r_c (1 + 1e-6), counting-sorted by cell
// (each cell's list then ordered by atom index, so the traversal is
// deterministic), and each centre scans the (2R+1)^3 stencil of cells around
// its own.  A candidate's image shift S follows from the stencil wrap and the
// two atoms' wrap counts, and the pair is kept iff the float64 displacement
//   off[x] = (S0*a[x] + S1*b[x]) + S2*c[x];  d[x] = (pos_j[x] + off[x]) - pos_i[x]
//   r2 = (d0*d0 + d1*d1) + d2*d2  <  r_c^2,   not (i == j and S == 0)
// evaluated with explicitly rounded operations (no contraction), i.e. the
// same rule the oracle applies to every candidate.  Counting pass, exclusive
// scan, fill pass: rows come out in ascending centre index.  A CSC index
// (edges grouped by neighbour j, ascending edge id) serves the force gather.
#include <cuda_runtime.h>

#include "internal.h"

namespace alg {

__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (out has n+1 entries; out[n] = total)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;   // elements per block (256 threads x 4)

__global__ void scan_block_kernel(const int* __restrict__ in, int* __restrict__ out, int n,
                                  int* __restrict__ block_sums) {
  __shared__ int warp_tot[8];
  const int base = blockIdx.x * kScanBlock;
  const int t = threadIdx.x;
  int v[4];
  int s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int idx = base + t * 4 + k;
    v[k] = (idx < n && in) ? in[idx] : 0;
    s += v[k];
  }
  // warp inclusive scan of per-thread sums
  int lane = t & 31, w = t >> 5;
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int wt = (lane < 8) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, wt, o);
      if (lane >= o) wt += y;
    }
    if (lane < 8) warp_tot[lane] = wt;
  }
  __syncthreads();
  int excl = x - s + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int idx = base + t * 4 + k;
    if (idx <= n) out[idx] = excl;
    excl += v[k];
  }
  if (t == 255 && block_sums) block_sums[blockIdx.x] = warp_tot[7];
}

__global__ void scan_add_kernel(int* __restrict__ out, int n, const int* __restrict__ block_pref) {
  const int base = blockIdx.x * kScanBlock;
  const int add = block_pref[blockIdx.x];
  for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
    int idx = base + k;
    if (idx <= n) out[idx] += add;
  }
}

size_t scan_tmp_bytes(int n) {
  size_t total = 0;
  int m = n + 1;
  while (m > 1) {
    int nb = (m + kScanBlock - 1) / kScanBlock;
    total += (size_t)(nb + 1) * 2 * sizeof(int) + 256;
    m = nb;
  }
  return total + 256;
}

// Scans in[0..n) into out[0..n] (out[n] = total); in == nullptr means zeros.
static void scan_rec(const int* in, int* out, int n, char* tmp, cudaStream_t st) {
  int nb = (n + 1 + kScanBlock - 1) / kScanBlock;
  if (nb == 1) {
    scan_block_kernel<<<1, 256, 0, st>>>(in, out, n, nullptr);
    return;
  }
  int* sums = reinterpret_cast<int*>(tmp);
  int* pref = sums + (nb + 1);
  char* next = reinterpret_cast<char*>(pref + (nb + 1)) + 256;
  scan_block_kernel<<<nb, 256, 0, st>>>(in, out, n, sums);
  scan_rec(sums, pref, nb, next, st);
  scan_add_kernel<<<nb, 256, 0, st>>>(out, n, pref);
}

void exclusive_scan_i32(const int* in, int* out, int n, int* d_total, void* tmp, size_t tmp_bytes,
                        cudaStream_t st) {
  (void)tmp_bytes;
  scan_rec(in, out, n, reinterpret_cast<char*>(tmp), st);
  if (d_total) cudaMemcpyAsync(d_total, out + n, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

// ---------------------------------------------------------------------------
// binning
// ---------------------------------------------------------------------------
__device__ __forceinline__ void frac_of(const double* p, const double* inv, double f[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = p[0] * inv[0 * 3 + k] + p[1] * inv[1 * 3 + k] + p[2] * inv[2 * 3 + k];
}

// monotone map double -> unsigned long long for atomic min/max
__device__ __forceinline__ unsigned long long dkey(double x) {
  unsigned long long b = __double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void minmax_frac_kernel(const double* __restrict__ pos, int n, CellGrid g,
                                   unsigned long long* __restrict__ mm) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double f[3];
    frac_of(pos + 3 * (size_t)i, g.inv, f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = fmin(lo[k], f[k]);
      hi[k] = fmax(hi[k], f[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&mm[k], dkey(lo[k]));
      atomicMax(&mm[3 + k], dkey(hi[k]));
    }
  }
}

__global__ void minmax_init_kernel(unsigned long long* mm) {
  int k = threadIdx.x;
  if (k < 3) mm[k] = ~0ull;
  else if (k < 6) mm[k] = 0ull;
}

__global__ void minmax_decode_kernel(const unsigned long long* mm, double* out) {
  int k = threadIdx.x;
  if (k < 6) {
    unsigned long long b = mm[k];
    b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
    out[k] = __longlong_as_double((long long)b);
  }
}

void nb_minmax_frac(const double* pos, int n, const double* inv, double* d_minmax, cudaStream_t st) {
  CellGrid g{};
  for (int k = 0; k < 9; ++k) g.inv[k] = inv[k];
  unsigned long long* mm = reinterpret_cast<unsigned long long*>(d_minmax + 6);
  minmax_init_kernel<<<1, 32, 0, st>>>(mm);
  int blocks = (n + 255) / 256;
  if (blocks > 1184) blocks = 1184;
  if (blocks < 1) blocks = 1;
  minmax_frac_kernel<<<blocks, 256, 0, st>>>(pos, n, g, mm);
  minmax_decode_kernel<<<1, 32, 0, st>>>(mm, d_minmax);
}

__global__ void bin_kernel(const double* __restrict__ pos, int n, CellGrid g, int* __restrict__ cell_of,
                           int* __restrict__ wrap, int* __restrict__ cell_count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[3];
  frac_of(pos + 3 * (size_t)i, g.inv, f);
  int c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double x;
    int w = 0;
    if (g.pbc[k]) {
      double fl = floor(f[k]);
      w = (int)fl;
      x = f[k] - fl;
    } else {
      x = (g.span[k] > 0) ? (f[k] - g.lo[k]) / g.span[k] : 0.0;
    }
    int ck = (int)floor(x * g.n[k]);
    ck = ck < 0 ? 0 : (ck >= g.n[k] ? g.n[k] - 1 : ck);
    c[k] = ck;
    wrap[3 * (size_t)i + k] = w;
  }
  int id = (c[0] * g.n[1] + c[1]) * g.n[2] + c[2];
  cell_of[i] = id;
  atomicAdd(&cell_count[id], 1);
}

void nb_bin(const double* pos, int n, const CellGrid& g, int* cell_of, int* wrap, int* cell_count,
            cudaStream_t st) {
  if (n <= 0) return;
  bin_kernel<<<(n + 255) / 256, 256, 0, st>>>(pos, n, g, cell_of, wrap, cell_count);
}

__global__ void place_kernel(const int* __restrict__ cell_of, int n, const int* __restrict__ cell_start,
                             int* __restrict__ cursor, int* __restrict__ sorted) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell_of[i];
  int k = atomicAdd(&cursor[c], 1);
  sorted[cell_start[c] + k] = i;
}

void nb_place(const int* cell_of, int n, const int* cell_start, int* cell_cursor, int* sorted,
              cudaStream_t st) {
  if (n <= 0) return;
  place_kernel<<<(n + 255) / 256, 256, 0, st>>>(cell_of, n, cell_start, cell_cursor, sorted);
}

// insertion sort of each segment [start[s], start[s+1]) (segments are short)
__global__ void sort_segments_kernel(const int* __restrict__ start, int nseg, int* __restrict__ v) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int b = start[s], e = start[s + 1];
  for (int x = b + 1; x < e; ++x) {
    int key = v[x];
    int y = x - 1;
    while (y >= b && v[y] > key) {
      v[y + 1] = v[y];
      --y;
    }
    v[y + 1] = key;
  }
}

void nb_sort_cells(const int* cell_start, int n_cells, int* sorted, cudaStream_t st) {
  if (n_cells <= 0) return;
  sort_segments_kernel<<<(n_cells + 255) / 256, 256, 0, st>>>(cell_start, n_cells, sorted);
}

void nb_sort_columns(const int* col_ptr, int n, int* col_edge, cudaStream_t st) {
  if (n <= 0) return;
  sort_segments_kernel<<<(n + 255) / 256, 256, 0, st>>>(col_ptr, n, col_edge);
}

// ---------------------------------------------------------------------------
// exact pair test (float64, explicitly rounded, no contraction)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool pair_test(const double* __restrict__ pi, const double* __restrict__ pj,
                                          const double* cell, int S0, int S1, int S2, double rc2,
                                          double d[3]) {
  double s0 = (double)S0, s1 = (double)S1, s2 = (double)S2;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    double off = __dadd_rn(__dadd_rn(__dmul_rn(s0, cell[0 * 3 + x]), __dmul_rn(s1, cell[1 * 3 + x])),
                           __dmul_rn(s2, cell[2 * 3 + x]));
    d[x] = __dsub_rn(__dadd_rn(pj[x], off), pi[x]);
  }
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < rc2;
}

// ---------------------------------------------------------------------------
// Verlet-skin reuse: the exact list of the current positions, filtered from a
// candidate list built at r_c + skin (every pair now within r_c was within
// r_c + skin at the build while no atom has moved skin/2 since).  One warp per
// centre row: each lane takes candidates of the row, applies the exact rule
// (pair_test, the pair's cutoff when a table is set), the warp counts the
// kept ones with a ballot (count pass) or writes them in candidate order at
// the row's offset (fill pass).
// ---------------------------------------------------------------------------
template <bool fill>
__global__ void skin_filter_kernel(const double* __restrict__ pos, int n, const double* __restrict__ cellp,
                                   const int* __restrict__ sk_row, const int* __restrict__ sk_j,
                                   const int* __restrict__ sk_S, double rc2, const double* __restrict__ pair_rc2,
                                   const int* __restrict__ species, int ns, int* __restrict__ count,
                                   const int* __restrict__ row_ptr, int* __restrict__ ej, int* __restrict__ ei,
                                   int* __restrict__ eS, double* __restrict__ ed) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  double cell[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) cell[q] = cellp[q];
  const double pi[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
  const int zi = pair_rc2 ? species[i] : 0;
  const int b = sk_row[i], e1 = sk_row[i + 1];
  int out = fill ? row_ptr[i] : 0;
  for (int e0 = b; e0 < e1; e0 += 32) {
    const int e = e0 + lane;
    bool keep = false;
    int j = 0, S0 = 0, S1 = 0, S2 = 0;
    double d[3] = {0.0, 0.0, 0.0};
    if (e < e1) {
      j = sk_j[e];
      S0 = sk_S[3 * (size_t)e]; S1 = sk_S[3 * (size_t)e + 1]; S2 = sk_S[3 * (size_t)e + 2];
      const double pj[3] = {pos[3 * (size_t)j], pos[3 * (size_t)j + 1], pos[3 * (size_t)j + 2]};
      const double r2c = pair_rc2 ? pair_rc2[zi * ns + species[j]] : rc2;
      keep = pair_test(pi, pj, cell, S0, S1, S2, r2c, d) && !(j == i && S0 == 0 && S1 == 0 && S2 == 0);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (fill && keep) {
      const int o = out + __popc(m & ((1u << lane) - 1u));
      ej[o] = j;
      ei[o] = i;
      eS[3 * (size_t)o] = S0; eS[3 * (size_t)o + 1] = S1; eS[3 * (size_t)o + 2] = S2;
      ed[3 * (size_t)o] = d[0]; ed[3 * (size_t)o + 1] = d[1]; ed[3 * (size_t)o + 2] = d[2];
    }
    out += __popc(m);
  }
  if (!fill && lane == 0) count[i] = out;
}

void nb_skin_filter(bool fill, const double* pos, int n, const double* d_cell, const int* sk_row, const int* sk_j,
                    const int* sk_S, double rc2, const double* pair_rc2, const int* species, int ns, int* count,
                    const int* row_ptr, int* ej, int* ei, int* eS, double* ed, cudaStream_t st) {
  if (n <= 0) return;
  const int threads = 256, blocks = (int)(((int64_t)n * 32 + threads - 1) / threads);
  if (fill)
    skin_filter_kernel<true><<<blocks, threads, 0, st>>>(pos, n, d_cell, sk_row, sk_j, sk_S, rc2, pair_rc2, species,
                                                         ns, count, row_ptr, ej, ei, eS, ed);
  else
    skin_filter_kernel<false><<<blocks, threads, 0, st>>>(pos, n, d_cell, sk_row, sk_j, sk_S, rc2, pair_rc2,
                                                          species, ns, count, row_ptr, ej, ei, eS, ed);
}

// Largest squared displacement of any atom since the reference positions, as
// the bits of a non-negative double (their order is the values' order).
__global__ void max_disp2_kernel(const double* __restrict__ pos, const double* __restrict__ ref, int n,
                                 unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    const double dx = pos[3 * (size_t)i] - ref[3 * (size_t)i], dy = pos[3 * (size_t)i + 1] - ref[3 * (size_t)i + 1],
                 dz = pos[3 * (size_t)i + 2] - ref[3 * (size_t)i + 2];
    v = dx * dx + dy * dy + dz * dz;
    if (!(v == v)) v = 1e300;   // a NaN position forces a rebuild (which then reports it)
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

void nb_max_disp2(const double* pos, const double* ref, int n, unsigned long long* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (n <= 0) return;
  max_disp2_kernel<<<(n + 255) / 256, 256, 0, st>>>(pos, ref, n, out);
}

// Wrapped positions pw = pos - wrap . cell in cell-sorted order (pos4[s] and
// pw[3 s ..] belong to atom sorted[s]): float32 for the prefilter, float64 for
// the displacements of accepted edges.
__global__ void pos4_kernel(const double* __restrict__ pos, const int* __restrict__ species, int n, CellGrid g,
                            const int* __restrict__ wrap, const int* __restrict__ sorted,
                            float4* __restrict__ pos4, double* __restrict__ pw, int4* __restrict__ wraps) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int j = sorted[s];
  double p[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    p[x] = pos[3 * (size_t)j + x];
#pragma unroll
    for (int k = 0; k < 3; ++k) p[x] -= (double)wrap[3 * (size_t)j + k] * g.cell[k * 3 + x];
  }
  pos4[s] = make_float4((float)p[0], (float)p[1], (float)p[2], __int_as_float(species[j]));
  pw[3 * (size_t)s] = p[0];
  pw[3 * (size_t)s + 1] = p[1];
  pw[3 * (size_t)s + 2] = p[2];
  wraps[s] = make_int4(wrap[3 * (size_t)j], wrap[3 * (size_t)j + 1], wrap[3 * (size_t)j + 2], 0);
}

// Neighbour search.  A float32 prefilter on the wrapped positions decides
// every candidate whose squared distance is farther than `band` from r_c^2;
// candidates inside the band take the exact float64 test.  `band` is computed
// on the host from a bound on the float32 rounding of the wrapped coordinates
// and image offsets (with a safety factor), so the prefilter never changes a
// decision.  Accepted edges get their float64 displacement for later stages:
// from the exact test inside the band, else (pw_j + q . cell) - pw_i from the
// float64 wrapped positions (the same vector up to float64 rounding; the
// edge's image shift is S = q - w_j + w_i).
// The fill pass writes through shared memory: a lane records each accepted
// candidate of its row (cell-order index s, image q, whether it took the exact
// test) in its warp's staging area, then the warp writes the 32 rows one after
// another with its lanes on consecutive edges of a row, so each store covers
// consecutive addresses (a row per lane would scatter every store over 32
// rows).  Edges past kFillStage in a row are written by their lane directly.
constexpr int kSearchThreads = 128;
constexpr int kFillStage = 32;

// The displacement of pair_test (the same float64 operations in the same order).
__device__ __forceinline__ void pair_disp(const double* __restrict__ pi, const double* __restrict__ pj,
                                          const double* cell, int S0, int S1, int S2, double d[3]) {
  double s0 = (double)S0, s1 = (double)S1, s2 = (double)S2;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    double off = __dadd_rn(__dadd_rn(__dmul_rn(s0, cell[0 * 3 + x]), __dmul_rn(s1, cell[1 * 3 + x])),
                           __dmul_rn(s2, cell[2 * 3 + x]));
    d[x] = __dsub_rn(__dadd_rn(pj[x], off), pi[x]);
  }
}

// image q (three signed 9-bit fields) and the exact-test flag of a staged edge
__device__ __forceinline__ int pack_q(int q0, int q1, int q2, bool exact) {
  return (q0 & 511) | ((q1 & 511) << 9) | ((q2 & 511) << 18) | (exact ? (1 << 27) : 0);
}
__device__ __forceinline__ int unpack_q(int v, int f) { return ((v >> (9 * f)) << 23) >> 23; }

template <bool fill>
__global__ void __launch_bounds__(kSearchThreads) search_kernel(
    const double* __restrict__ pos, int n, CellGrid g, const int* __restrict__ cell_of,
    const int4* __restrict__ wraps, const int* __restrict__ cell_start, const int* __restrict__ sorted,
    const float4* __restrict__ pos4, const double* __restrict__ pw, double rc2, float band,
    const double* __restrict__ pair_rc2, int ns, int* __restrict__ count, const int* __restrict__ row_ptr,
    int* __restrict__ ej, int* __restrict__ ei, int* __restrict__ eS, double* __restrict__ ed,
    int* __restrict__ d_err) {
  __shared__ int2 stage[fill ? kSearchThreads : 1][fill ? kFillStage : 1];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = t < n;
  const int i = act ? sorted[t] : 0;
  if (act && i >= g.n_centres) {   // ghost atoms (spatial decomposition) are neighbours only, never centres
    if (!fill) count[i] = 0;
    act = false;
  }
  if constexpr (!fill) {
    if (!act) return;
  }
  int4 wi = make_int4(0, 0, 0, 0);
  double pi[3] = {0.0, 0.0, 0.0}, pwi[3] = {0.0, 0.0, 0.0};
  int k = 0, base = 0, cap = 0;
  if (act) {
    const int ci = cell_of[i];
    int c[3];
    c[2] = ci % g.n[2];
    c[1] = (ci / g.n[2]) % g.n[1];
    c[0] = ci / (g.n[2] * g.n[1]);
    wi = wraps[t];   // cell-order copies of the wrap counts: coalesced with pos4
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      pi[x] = pos[3 * (size_t)i + x];
      pwi[x] = pw[3 * (size_t)t + x];
    }
    const float4 pi4 = pos4[t];
    const float rc2f = (float)rc2;
    const float lo2 = rc2f - band, hi2 = rc2f + band;
    // per-ordered-pair cutoffs: row of the centre's species (the band of the largest
    // cutoff bounds the float32 error of every smaller one)
    const double* prow = pair_rc2 ? pair_rc2 + (size_t)__float_as_int(pi4.w) * ns : nullptr;
    float cf[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) cf[q] = (float)g.cell[q];
    base = fill ? row_ptr[i] : 0;
    cap = fill ? (row_ptr[i + 1] - base) : 0;
    for (int d0 = -g.R[0]; d0 <= g.R[0]; ++d0) {
      int cc0 = c[0] + d0, q0 = 0;
      if (g.pbc[0]) { q0 = floordiv(cc0, g.n[0]); cc0 -= q0 * g.n[0]; }
      else if (cc0 < 0 || cc0 >= g.n[0]) continue;
      for (int d1 = -g.R[1]; d1 <= g.R[1]; ++d1) {
        int cc1 = c[1] + d1, q1 = 0;
        if (g.pbc[1]) { q1 = floordiv(cc1, g.n[1]); cc1 -= q1 * g.n[1]; }
        else if (cc1 < 0 || cc1 >= g.n[1]) continue;
        for (int d2 = -g.R[2]; d2 <= g.R[2]; ++d2) {
          int cc2 = c[2] + d2, q2 = 0;
          if (g.pbc[2]) { q2 = floordiv(cc2, g.n[2]); cc2 -= q2 * g.n[2]; }
          else if (cc2 < 0 || cc2 >= g.n[2]) continue;
          const int cell = (cc0 * g.n[1] + cc1) * g.n[2] + cc2;
          const int b = cell_start[cell], e = cell_start[cell + 1];
          // image offset of this stencil cell (float32), relative to i
          const float ox = (float)q0 * cf[0] + (float)q1 * cf[3] + (float)q2 * cf[6] - pi4.x;
          const float oy = (float)q0 * cf[1] + (float)q1 * cf[4] + (float)q2 * cf[7] - pi4.y;
          const float oz = (float)q0 * cf[2] + (float)q1 * cf[5] + (float)q2 * cf[8] - pi4.z;
          for (int s = b; s < e; ++s) {
            const float4 pj = pos4[s];
            const float dx = pj.x + ox, dy = pj.y + oy, dz = pj.z + oz;
            const float r2f = dx * dx + dy * dy + dz * dz;
            if (r2f > hi2) continue;
            double rc2p = rc2;
            float lo2p = lo2;
            if (prow) {
              rc2p = prow[__float_as_int(pj.w)];
              const float rc2pf = (float)rc2p;
              if (r2f > rc2pf + band) continue;
              lo2p = rc2pf - band;
            }
            const int4 wj = wraps[s];
            const int S0 = g.pbc[0] ? q0 - wj.x + wi.x : 0;
            const int S1 = g.pbc[1] ? q1 - wj.y + wi.y : 0;
            const int S2 = g.pbc[2] ? q2 - wj.z + wi.z : 0;
            if (s == t && S0 == 0 && S1 == 0 && S2 == 0) continue;   // (s = t: j = i)
            const bool exact = r2f >= lo2p;
            double d[3];
            if (exact && !pair_test(pi, pos + 3 * (size_t)sorted[s], g.cell, S0, S1, S2, rc2p, d)) continue;
            if constexpr (fill) {
              if (k < kFillStage) {
                stage[threadIdx.x][k] = make_int2(s, pack_q(q0, q1, q2, exact));
              } else if (k < cap) {
                // past the staging area: this lane writes the edge itself
                if (!exact) {
#pragma unroll
                  for (int x = 0; x < 3; ++x) {
                    const double qoff = (q0 | q1 | q2) ? ((double)q0 * g.cell[x] + (double)q1 * g.cell[3 + x]) +
                                                             (double)q2 * g.cell[6 + x]
                                                       : 0.0;
                    d[x] = (pw[3 * (size_t)s + x] + qoff) - pwi[x];
                  }
                }
                const size_t o = (size_t)base + k;
                ej[o] = sorted[s];
                ei[o] = i;
                eS[3 * o] = S0; eS[3 * o + 1] = S1; eS[3 * o + 2] = S2;
                ed[3 * o] = d[0]; ed[3 * o + 1] = d[1]; ed[3 * o + 2] = d[2];
              }
            }
            ++k;
          }
        }
      }
    }
  }
  if constexpr (!fill) {
    count[i] = k;
  } else {
    if (act && k != cap) atomicOr(d_err, kErrNeighbor);
    __syncwarp();
    // the warp's rows one after another, lanes on consecutive edges
    const int lane = threadIdx.x & 31, w0 = threadIdx.x & ~31;
    const int nst = act ? min(min(k, cap), kFillStage) : 0;
    for (int r = 0; r < 32; ++r) {
      const int nr = __shfl_sync(0xffffffffu, nst, r);
      if (nr == 0) continue;
      const int ir = __shfl_sync(0xffffffffu, i, r);
      const int br = __shfl_sync(0xffffffffu, base, r);
      const int wx = __shfl_sync(0xffffffffu, wi.x, r), wy = __shfl_sync(0xffffffffu, wi.y, r),
                wz = __shfl_sync(0xffffffffu, wi.z, r);
      double pir[3], pwr[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        pir[x] = __shfl_sync(0xffffffffu, pi[x], r);
        pwr[x] = __shfl_sync(0xffffffffu, pwi[x], r);
      }
      for (int kk = lane; kk < nr; kk += 32) {
        const int2 en = stage[w0 + r][kk];
        const int s = en.x;
        const int q0 = unpack_q(en.y, 0), q1 = unpack_q(en.y, 1), q2 = unpack_q(en.y, 2);
        const bool exact = (en.y >> 27) & 1;
        const int j = sorted[s];
        const int4 wj = wraps[s];
        const int S0 = g.pbc[0] ? q0 - wj.x + wx : 0;
        const int S1 = g.pbc[1] ? q1 - wj.y + wy : 0;
        const int S2 = g.pbc[2] ? q2 - wj.z + wz : 0;
        double d[3];
        if (exact) {
          pair_disp(pir, pos + 3 * (size_t)j, g.cell, S0, S1, S2, d);
        } else {
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const double qoff = (q0 | q1 | q2) ? ((double)q0 * g.cell[x] + (double)q1 * g.cell[3 + x]) +
                                                     (double)q2 * g.cell[6 + x]
                                               : 0.0;
            d[x] = (pw[3 * (size_t)s + x] + qoff) - pwr[x];
          }
        }
        const size_t o = (size_t)br + kk;
        ej[o] = j;
        ei[o] = ir;
        eS[3 * o] = S0; eS[3 * o + 1] = S1; eS[3 * o + 2] = S2;
        ed[3 * o] = d[0]; ed[3 * o + 1] = d[1]; ed[3 * o + 2] = d[2];
      }
    }
  }
}

void nb_pos4(const double* pos, const int* species, int n, const CellGrid& g, const int* wrap, const int* sorted,
             float4* pos4, double* pw, int4* wraps, cudaStream_t st) {
  if (n <= 0) return;
  pos4_kernel<<<(n + 255) / 256, 256, 0, st>>>(pos, species, n, g, wrap, sorted, pos4, pw, wraps);
}

void nb_search(bool fill, const double* pos, int n, const CellGrid& g, const int* cell_of,
               const int4* wraps, const int* cell_start, const int* sorted, const float4* pos4, const double* pw,
               double rc2, float band, const double* pair_rc2, int ns, int* count, const int* row_ptr, int* ej,
               int* ei, int* eS, double* ed, int* d_err, cudaStream_t st) {
  if (n <= 0) return;
  if (fill)
    search_kernel<true><<<(n + kSearchThreads - 1) / kSearchThreads, kSearchThreads, 0, st>>>(pos, n, g, cell_of, wraps, cell_start, sorted, pos4, pw, rc2,
                                                         band, pair_rc2, ns, count, row_ptr, ej, ei, eS, ed, d_err);
  else
    search_kernel<false><<<(n + kSearchThreads - 1) / kSearchThreads, kSearchThreads, 0, st>>>(pos, n, g, cell_of, wraps, cell_start, sorted, pos4, pw, rc2,
                                                          band, pair_rc2, ns, count, row_ptr, ej, ei, eS, ed, d_err);
}

// ---------------------------------------------------------------------------
// batched structures: all pairs of each structure over its image range
// ---------------------------------------------------------------------------
__global__ void brute_batched_kernel(bool fill, const double* __restrict__ pos,
                                     const int64_t* __restrict__ offs, const double* __restrict__ cells,
                                     const int* __restrict__ pbc, const int* __restrict__ nimg,
                                     double rc2, const int* __restrict__ species,
                                     const double* __restrict__ pair_rc2, int ns,
                                     const int* __restrict__ atom_struct, int n,
                                     int* __restrict__ count, const int* __restrict__ row_ptr,
                                     int* __restrict__ ej, int* __restrict__ ei, int* __restrict__ eS,
                                     double* __restrict__ ed, int* __restrict__ d_err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = atom_struct[i];
  const int j0 = (int)offs[b], j1 = (int)offs[b + 1];
  double zero_cell[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const double* cell = cells ? cells + 9 * (size_t)b : zero_cell;
  int nI[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) nI[k] = (cells && pbc[3 * b + k]) ? nimg[3 * b + k] : 0;
  double pi[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
  int k = 0;
  const int base = fill ? row_ptr[i] : 0;
  const int cap = fill ? (row_ptr[i + 1] - base) : 0;
  const double* prow = pair_rc2 ? pair_rc2 + (size_t)species[i] * ns : nullptr;
  for (int j = j0; j < j1; ++j) {
    const double rc2p = prow ? prow[species[j]] : rc2;   // the ordered pair's cutoff
    for (int S0 = -nI[0]; S0 <= nI[0]; ++S0)
      for (int S1 = -nI[1]; S1 <= nI[1]; ++S1)
        for (int S2 = -nI[2]; S2 <= nI[2]; ++S2) {
          if (j == i && S0 == 0 && S1 == 0 && S2 == 0) continue;
          double d[3];
          if (!pair_test(pi, pos + 3 * (size_t)j, cell, S0, S1, S2, rc2p, d)) continue;
          if (fill && k < cap) {
            size_t o = (size_t)base + k;
            ej[o] = j;
            ei[o] = i;
            eS[3 * o] = S0; eS[3 * o + 1] = S1; eS[3 * o + 2] = S2;
            ed[3 * o] = d[0]; ed[3 * o + 1] = d[1]; ed[3 * o + 2] = d[2];
          }
          ++k;
        }
  }
  if (fill) {
    if (k != cap) atomicOr(d_err, kErrNeighbor);
  } else {
    count[i] = k;
  }
}

void nb_bruteforce_batched(bool fill, const double* pos, const int64_t* offs, int nstruct,
                           const double* cells, const int* pbc, const int* nimg, double rc2,
                           const int* species, const double* pair_rc2, int ns,
                           const int* atom_struct, int n, int* count, const int* row_ptr, int* ej,
                           int* ei, int* eS, double* ed, int* d_err, cudaStream_t st) {
  (void)nstruct;
  if (n <= 0) return;
  brute_batched_kernel<<<(n + 127) / 128, 128, 0, st>>>(fill, pos, offs, cells, pbc, nimg, rc2, species, pair_rc2,
                                                        ns, atom_struct, n, count, row_ptr, ej, ei, eS, ed,
                                                        d_err);
}

// Per structure: spread (max - min) of the fractional coordinates, so the
// image range covers positions that are not wrapped into the cell.
__global__ void struct_span_kernel(const double* __restrict__ pos, const int64_t* __restrict__ offs,
                                   const double* __restrict__ inv, double* __restrict__ span) {
  const int b = blockIdx.x;
  __shared__ double lo[3][128], hi[3][128];
  double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
  for (long long i = offs[b] + threadIdx.x; i < offs[b + 1]; i += blockDim.x) {
    double f[3];
    frac_of(pos + 3 * i, inv + 9 * (size_t)b, f);
    for (int k = 0; k < 3; ++k) { l[k] = fmin(l[k], f[k]); h[k] = fmax(h[k], f[k]); }
  }
  for (int k = 0; k < 3; ++k) { lo[k][threadIdx.x] = l[k]; hi[k][threadIdx.x] = h[k]; }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) {
        lo[k][threadIdx.x] = fmin(lo[k][threadIdx.x], lo[k][threadIdx.x + s]);
        hi[k][threadIdx.x] = fmax(hi[k][threadIdx.x], hi[k][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    double sp = hi[threadIdx.x][0] - lo[threadIdx.x][0];
    span[3 * b + threadIdx.x] = (sp > 0) ? sp : 0.0;
  }
}

void nb_struct_span(const double* pos, const int64_t* offs, const double* inv, int nstruct, double* span,
                    cudaStream_t st) {
  if (nstruct <= 0) return;
  struct_span_kernel<<<nstruct, 128, 0, st>>>(pos, offs, inv, span);
}

// ---------------------------------------------------------------------------
// CSC index: edges grouped by neighbour atom j
// ---------------------------------------------------------------------------
__global__ void col_count_kernel(const int* __restrict__ ej, int E, int* __restrict__ col_count) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E) atomicAdd(&col_count[ej[e]], 1);
}

void nb_columns(const int* ej, int E, int n, int* col_count, cudaStream_t st) {
  (void)n;
  if (E <= 0) return;
  col_count_kernel<<<(E + 255) / 256, 256, 0, st>>>(ej, E, col_count);
}

__global__ void col_fill_kernel(const int* __restrict__ ej, int E, const int* __restrict__ col_ptr,
                                int* __restrict__ cursor, int* __restrict__ col_edge) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int j = ej[e];
  int k = atomicAdd(&cursor[j], 1);
  col_edge[col_ptr[j] + k] = e;
}

void nb_fill_columns(const int* ej, int E, const int* col_ptr, int* cursor, int* col_edge,
                     cudaStream_t st) {
  if (E <= 0) return;
  col_fill_kernel<<<(E + 255) / 256, 256, 0, st>>>(ej, E, col_ptr, cursor, col_edge);
}

}  // namespace alg
