// Host orchestration and the C ABI of liballegro_gb300 (include/allegro.h).
//
// The context owns the model (weights on the device as float32 and bfloat16,
// forward and transposed), the tensor-product constants, and a device arena:
// per-atom and per-edge arrays of the neighbour list, and a chunk workspace
// for the per-edge activations.  Edges are evaluated in chunks of whole CSR
// rows (every centre atom's environment sum is complete inside one chunk, the
// strict locality of Eq. 1), so the activation working set is bounded by the
// chunk size, not by the system size.
//
// One evaluation (Sec. "Allegro", Fig. "architecture"):
//   geometry/basis -> two-body MLP -> [embedding | env weights 1]
//   -> per layer: row kernel (environment sum, tensor product, scalars)
//      -> latent MLP -> env weights of the next layer
//   -> edge energy (linear edge MLP folded into one vector)
// and the hand-written adjoint in reverse order down to dE/dd_e, then the
// float64 per-atom reduction (energies, forces by row/column gathers, virial).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

using namespace alg;

namespace {

inline int pad8(int x) { return (x + 7) / 8 * 8; }
inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// ------------------------------------------------------------------------
// small kernels
// ------------------------------------------------------------------------
__global__ void map_types_kernel(const int* __restrict__ types, const double* __restrict__ pos, int n,
                                 const int* __restrict__ map, int nmap, int* __restrict__ species,
                                 int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t = types[i];
  bool bad = (t < 0 || t >= nmap);
  int s = bad ? 0 : map[t];
  if (s < 0) bad = true;
  double x = pos[3 * (size_t)i], y = pos[3 * (size_t)i + 1], z = pos[3 * (size_t)i + 2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) bad = true;
  if (bad) atomicOr(err, kErrBadInput);
  species[i] = bad ? 0 : s;
}

__global__ void atom_struct_kernel(const int64_t* __restrict__ offs, int nstruct, int* __restrict__ atom_struct) {
  int b = blockIdx.x;
  if (b >= nstruct) return;
  for (long long i = offs[b] + threadIdx.x; i < offs[b + 1]; i += blockDim.x) atom_struct[i] = b;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Per-launch timing of the library's kernels (CUDA events on the launching
// stream) with the algorithmic FLOPs and bytes of each launch.
struct ProfRec {
  const char* name;
  int ev;
  double flops, bytes;
  int launches;
};
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;      // pairs: 2k = start, 2k+1 = stop
  std::vector<ProfRec> recs;
};

// Capacity (elements) of each growable device buffer.
struct Cap {
  int64_t v = 0;
};
struct Caps {
  Cap pos, types, species, row_ptr, col_ptr, count, cell_of, wrap, sorted, atom_struct, Eatom, F, Wat, pos4, pw, wraps;
  Cap ej, ei, eS, ed, col_edge, Ee, g;
  Cap cc, cs, ccur;
  Cap offs, cells, pbc, nimg, Eout, Wout;
};

}  // namespace

// --------------------------------------------------------------------------
// context
// --------------------------------------------------------------------------
struct allegro_ctx {
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  int prec = ALLEGRO_PREC_FP32;
  Arch arch;
  std::vector<int> species_map;
  std::string err;
  // per-ordered-species-pair cutoffs (arch.pair_basis / arch.pair_rc2 point here)
  float* d_pair_basis = nullptr;
  double* d_pair_rc2 = nullptr;
  float* d_zbl = nullptr;                  // ZBL pair table (arch.zbl points here)

  // model on the device
  std::vector<Lin> tb;                     // two-body layers
  Lin w01;                                 // [embedding ; env weights of layer 1]
  Lin env2;                                // env weights of layer 2 (two- and three-layer models)
  Lin env3;                                // env weights of layer 3 (three-layer models)
  // models the specialised row kernels do not take (three layers, or l_max 3): the
  // generic row path: the layer tensors' values in the kernels' order
  bool generic = false;
  std::vector<float> gen_vals;
  int gdim[kGenMaxLayers + 1] = {};
  std::vector<std::vector<Lin>> lat;       // latent MLP of layers 1..nl
  // BF16 path: the adjoint of x^{L-1} in one GEMM over [wbar^L | zbar^L] (K-concatenated):
  // B[n][k] = W_env^L[k][n] for k < K1, W_lat^L_0[k - K1][n] after; null when K1 % 64 != 0
  bf16* headB[kGenMaxLayers] = {nullptr, nullptr, nullptr};
  int headK1[kGenMaxLayers] = {0, 0, 0}, headK[kGenMaxLayers] = {0, 0, 0}, headLd[kGenMaxLayers] = {0, 0, 0};
  // FP8 path: E4M3 copies of the head maps ([Nx][headLd8] bytes) and their scales
  uint8_t* headB8[kGenMaxLayers] = {nullptr, nullptr, nullptr};
  int headLd8[kGenMaxLayers] = {0, 0, 0};
  float headS8[kGenMaxLayers] = {1.0f, 1.0f, 1.0f};
  // FP8 path: per-tensor amax slots (float bits) of the activations the E4M3 GEMMs read,
  // cleared at the start of every chunk
  unsigned* d_amax = nullptr;
  float* d_v = nullptr;                    // folded edge-energy vector
  double* d_sigma = nullptr;
  double* d_mu = nullptr;
  int* d_map = nullptr;
  int nmap = 0;
  TPConst tp{};
  std::vector<void*> weight_allocs;

  // state of the last neighbour build
  bool have_nb = false;
  int64_t n_atoms = 0, n_edges = 0;
  int64_t n_centres = 0;                   // atoms [0, n_centres) are centres (the rest are ghosts)
  int nstruct = 0;
  bool batched = false;
  std::vector<int> h_row_ptr;              // host copy of row_ptr (for chunking)

  // capacities and policy
  int64_t atom_cap = 0, edge_cap = 0;
  bool fixed = false;
  int64_t chunk_edges_user = 0;

  // per-atom arrays
  double* d_pos = nullptr;
  int* d_types = nullptr;
  int* d_species = nullptr;
  int* d_row_ptr = nullptr;
  int* d_col_ptr = nullptr;
  int* d_count = nullptr;
  int* d_cell_of = nullptr;
  int* d_wrap = nullptr;
  int* d_sorted = nullptr;
  float4* d_pos4 = nullptr;                // wrapped float32 positions in cell order
  int4* d_wraps = nullptr;                 // wrap counts in cell order
  double* d_pw = nullptr;                  // wrapped float64 positions in cell order [3 n]
  int* d_atom_struct = nullptr;
  double* d_Eatom = nullptr;
  double* d_F = nullptr;
  double* d_Wat = nullptr;
  // per-edge arrays
  int* d_ej = nullptr;
  int* d_ei = nullptr;
  int* d_eS = nullptr;
  double* d_ed = nullptr;
  int* d_col_edge = nullptr;
  float* d_Ee = nullptr;
  float* d_g = nullptr;
  // cells
  int* d_cell_count = nullptr;
  int* d_cell_start = nullptr;
  int* d_cell_cursor = nullptr;
  int64_t cell_cap = 0;
  // structures
  int64_t* d_offs = nullptr;
  double* d_cells = nullptr;
  int* d_pbc = nullptr;
  int* d_nimg = nullptr;
  double* d_Eout = nullptr;
  double* d_Wout = nullptr;
  int64_t struct_cap = 0;
  // scratch
  void* d_scan_tmp = nullptr;
  size_t scan_tmp_cap = 0;
  int* d_err = nullptr;
  int* d_total = nullptr;
  double* d_minmax = nullptr;
  double* d_red_scratch = nullptr;         // partial sums of the per-structure reduction
  Caps caps;
  Profiler prof;
  // velocity-Verlet state
  double* d_md_pos = nullptr;
  double* d_md_vel = nullptr;
  double* d_md_invm = nullptr;
  int* d_md_types = nullptr;
  double* d_md_masses = nullptr;
  double* d_md_E = nullptr;
  double* d_md_K = nullptr;
  double* d_md_part = nullptr;
  int64_t md_atoms = 0, md_steps = 0;
  // Verlet-skin neighbour reuse in allegro_md_verlet: candidate list at r_c + skin
  double md_skin = 0.0;
  int64_t md_rebuilds = 0;
  int* d_sk_row = nullptr;
  int* d_sk_j = nullptr;
  int* d_sk_S = nullptr;
  double* d_sk_ref = nullptr;              // positions at the candidate build
  double* d_cell9 = nullptr;               // cell of the last single-structure build (device copy)
  unsigned long long* d_maxd = nullptr;
  int64_t sk_row_cap = 0, sk_cap = 0, sk_S_cap = 0;
  double h_cell[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int64_t launches = 0;                    // kernel launches issued by this context
  // Launch configuration of the evaluation (set by the autotuner, or the defaults):
  // edges per chunk (0 = largest that fits), which layer pairs run as one fused
  // kernel (bit k = pair kind k, see pair_kind), epilogue warps per TMEM quarter
  // of the arithmetic single-GEMM epilogues (2 or 4)
  struct Tune {
    int64_t chunk_edges = 0;
    int chain_mask = 0x3f;
    int epq_wide = 4;
  } tune;
  int autotune = 0;                        // allegro_set_autotune
  struct TuneRec {
    Tune best;
    std::vector<std::pair<std::string, double>> trials;   // configuration, ms
  };
  std::map<std::string, TuneRec> tuned;    // shape bucket -> result
  // CUDA-graph replay of the evaluation (allegro_set_graphs)
  bool use_graphs = false;
  struct GraphKey {
    std::vector<int> bounds;
    std::vector<const void*> ptrs;
    int64_t n_atoms = -1, n_edges = -1;
    int nstruct = 0;
    bool backward = false;
    int64_t chunk = 0;
    int chain_mask = 0, epq = 0;
    cudaStream_t stream = nullptr;
    bool operator==(const GraphKey& o) const {
      return bounds == o.bounds && ptrs == o.ptrs && n_atoms == o.n_atoms && n_edges == o.n_edges &&
             nstruct == o.nstruct && backward == o.backward && chunk == o.chunk && chain_mask == o.chain_mask &&
             epq == o.epq && stream == o.stream;
    }
  };
  GraphKey graph_key, seen_key;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0;              // kernels in the captured graph
  int64_t graph_replays = 0;

  // chunk workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int64_t ws_edges = 0, ws_atoms = 0;
};

namespace {

// activations stored in bf16 (the BF16 and FP8 precisions)
bool bf16_storage(const allegro_ctx* c) { return c->prec == ALLEGRO_PREC_BF16 || c->prec == ALLEGRO_PREC_FP8; }

// power-of-two scale s with max|W| / s <= 448 (the largest E4M3 value)
float e4m3_weight_scale(double amax) {
  if (!(amax > 0.0)) return 1.0f;
  int e;
  const double m = frexp(amax / 448.0, &e);   // amax / 448 = m 2^e, m in [0.5, 1)
  return (float)ldexp(1.0, m == 0.5 ? e - 1 : e);
}

allegro_status fail(allegro_ctx* c, allegro_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                        \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      cudaGetLastError();                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? ALLEGRO_E_OOM : ALLEGRO_E_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                                  \
    }                                                                                              \
  } while (0)

template <typename T>
cudaError_t regrow(T*& p, int64_t& cap, int64_t need, double headroom = 1.05) {
  if (need <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  int64_t n = std::max<int64_t>((int64_t)(need * headroom) + 16, 16);
  cudaError_t e = cudaMalloc(&p, (size_t)n * sizeof(T));
  cap = (e == cudaSuccess) ? n : 0;
  return e;
}

template <typename T>
cudaError_t grow(T*& p, Cap& cap, int64_t need) {
  return regrow(p, cap.v, need);
}

inline Caps& caps_of(allegro_ctx* c) { return c->caps; }

int prof_begin(allegro_ctx* c, const char* name, double flops, double bytes, int launches) {
  c->launches += launches;
  if (!c->prof.on) return -1;
  Profiler& P = c->prof;
  int k = (int)P.recs.size();
  while ((int)P.ev.size() < 2 * (k + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    P.ev.push_back(e);
  }
  P.recs.push_back({name, k, flops, bytes, launches});
  cudaEventRecord(P.ev[2 * k], c->stream);
  return k;
}

void prof_end(allegro_ctx* c, int k) {
  if (k >= 0) cudaEventRecord(c->prof.ev[2 * k + 1], c->stream);
}

struct ProfScope {
  allegro_ctx* c;
  int k;
  ProfScope(allegro_ctx* c_, const char* name, double flops, double bytes, int launches = 1)
      : c(c_), k(prof_begin(c_, name, flops, bytes, launches)) {}
  ~ProfScope() { prof_end(c, k); }
};

// ------------------------------------------------------------------------
// weights
// ------------------------------------------------------------------------
struct Reader {
  const uint8_t* p;
  size_t n, off = 0;
  bool ok = true;
  template <typename T>
  T get() {
    T v{};
    if (off + sizeof(T) > n) { ok = false; return v; }
    memcpy(&v, p + off, sizeof(T));
    off += sizeof(T);
    return v;
  }
  bool arr_f32(std::vector<float>& out, size_t count) {
    if (off + count * 4 > n) { ok = false; return false; }
    out.resize(count);
    memcpy(out.data(), p + off, count * 4);
    off += count * 4;
    return true;
  }
  bool arr_f64(std::vector<double>& out, size_t count) {
    if (off + count * 8 > n) { ok = false; return false; }
    out.resize(count);
    memcpy(out.data(), p + off, count * 8);
    off += count * 8;
    return true;
  }
};

allegro_status upload_lin(allegro_ctx* c, const std::vector<float>& W, int N, int K, Lin& L) {
  L.N = N; L.K = K;
  L.ld = pad8(K);
  L.ldT = pad8(N);
  std::vector<float> f((size_t)N * L.ld, 0.0f), fT((size_t)K * L.ldT, 0.0f);
  std::vector<bf16> b((size_t)N * L.ld), bT((size_t)K * L.ldT);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      f[(size_t)n * L.ld + k] = W[(size_t)n * K + k];
      fT[(size_t)k * L.ldT + n] = W[(size_t)n * K + k];
    }
  for (size_t q = 0; q < f.size(); ++q) b[q] = __float2bfloat16_rn(f[q]);
  for (size_t q = 0; q < fT.size(); ++q) bT[q] = __float2bfloat16_rn(fT[q]);
  CUDA_TRY(c, cudaMalloc(&L.f32, f.size() * 4));
  c->weight_allocs.push_back(L.f32);
  CUDA_TRY(c, cudaMalloc(&L.f32T, fT.size() * 4));
  c->weight_allocs.push_back(L.f32T);
  CUDA_TRY(c, cudaMalloc(&L.b16, b.size() * 2));
  c->weight_allocs.push_back(L.b16);
  CUDA_TRY(c, cudaMalloc(&L.b16T, bT.size() * 2));
  c->weight_allocs.push_back(L.b16T);
  CUDA_TRY(c, cudaMemcpy(L.f32, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(L.f32T, fT.data(), fT.size() * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(L.b16, b.data(), b.size() * 2, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(L.b16T, bT.data(), bT.size() * 2, cudaMemcpyHostToDevice));
  if (c->prec == ALLEGRO_PREC_FP8) {
    // E4M3 copies with one power-of-two scale per tensor (W and its transpose share max|W|)
    double amax = 0.0;
    for (float x : W) amax = std::max(amax, (double)fabsf(x));
    L.s8 = L.s8T = e4m3_weight_scale(amax);
    L.ld8 = (K + 15) / 16 * 16;
    L.ld8T = (N + 15) / 16 * 16;
    CUDA_TRY(c, cudaMalloc(&L.f8, (size_t)N * L.ld8));
    c->weight_allocs.push_back(L.f8);
    CUDA_TRY(c, cudaMalloc(&L.f8T, (size_t)K * L.ld8T));
    c->weight_allocs.push_back(L.f8T);
    fp8_quantize(L.f32, N, K, L.ld, L.f8, L.ld8, 1.0f / L.s8, 0);
    fp8_quantize(L.f32T, K, N, L.ldT, L.f8T, L.ld8T, 1.0f / L.s8T, 0);
    CUDA_TRY(c, cudaDeviceSynchronize());
  }
  return ALLEGRO_OK;
}

allegro_status load_model(allegro_ctx* c, const void* blob, size_t bytes) {
  Reader r{reinterpret_cast<const uint8_t*>(blob), bytes};
  if (bytes < 8 || memcmp(blob, "ALGW", 4) != 0) return fail(c, ALLEGRO_E_INVALID, "weights: bad magic");
  r.off = 4;
  uint32_t ver = r.get<uint32_t>();
  if (ver != 1) return fail(c, ALLEGRO_E_INVALID, "weights: unsupported version %u", ver);
  Arch& a = c->arch;
  a.rc = r.get<double>();
  a.ann = r.get<double>();
  a.ns = r.get<int32_t>(); a.nb = r.get<int32_t>(); a.p = r.get<int32_t>(); a.lmax = r.get<int32_t>();
  a.nl = r.get<int32_t>(); a.C = r.get<int32_t>();
  int n2 = r.get<int32_t>(), nlat = r.get<int32_t>(), ned = r.get<int32_t>();
  if (!r.ok || n2 < 1 || n2 > 16 || nlat < 1 || nlat > 16 || ned < 0 || ned > 16)
    return fail(c, ALLEGRO_E_INVALID, "weights: bad header");
  for (int k = 0; k < n2; ++k) a.tb.push_back(r.get<int32_t>());
  for (int k = 0; k < nlat; ++k) a.lat.push_back(r.get<int32_t>());
  for (int k = 0; k < ned; ++k) a.edge.push_back(r.get<int32_t>());
  if (!r.ok) return fail(c, ALLEGRO_E_INVALID, "weights: truncated header");
  if (a.nl < 1 || a.nl > kGenMaxLayers)
    return fail(c, ALLEGRO_E_INVALID, "weights: %d layers (supported: 1 to 3)", a.nl);
  if (a.lmax < 1 || a.lmax > kMaxLmax) return fail(c, ALLEGRO_E_INVALID, "weights: l_max %d (supported: 1 to 3)", a.lmax);
  c->generic = (a.nl > 2 || a.lmax > 2 || c->prec == ALLEGRO_PREC_FP8);
  a.generic = c->generic;
  if (a.C < 8 || a.C > kMaxChannels || (a.C & (a.C - 1)))
    return fail(c, ALLEGRO_E_INVALID, "weights: %d channels (supported: powers of two 8..128)", a.C);
  if (a.ns < 1 || a.ns > kMaxSpecies || a.nb < 1 || a.nb > kMaxBessel || a.p < 2 || a.p > 16 || !(a.rc > 0) ||
      !(a.ann > 0))
    return fail(c, ALLEGRO_E_INVALID, "weights: bad species/basis/cutoff fields");
  for (int w : a.tb) if (w < 1 || w > kMaxWidth) return fail(c, ALLEGRO_E_INVALID, "weights: bad two-body width");
  for (int w : a.lat) if (w < 1 || w > kMaxWidth) return fail(c, ALLEGRO_E_INVALID, "weights: bad latent width");
  for (int w : a.edge) if (w < 1 || w > 4096) return fail(c, ALLEGRO_E_INVALID, "weights: bad edge width");

  const int nw = a.n_w();
  std::vector<std::vector<float>> Wtb(n2);
  int fan = a.K0in();
  for (int k = 0; k < n2; ++k) {
    r.arr_f32(Wtb[k], (size_t)a.tb[k] * fan);
    fan = a.tb[k];
  }
  std::vector<float> Wemb;
  r.arr_f32(Wemb, (size_t)nw * a.tb.back());
  const int lm = a.lmax + 1;
  std::vector<std::vector<float>> Wenv(a.nl), theta(a.nl);
  std::vector<std::vector<std::vector<float>>> Wlat(a.nl, std::vector<std::vector<float>>(nlat));
  for (int L = 1; L <= a.nl; ++L) {
    int kin = a.Klat(L - 1);
    r.arr_f32(Wenv[L - 1], (size_t)nw * kin);
    r.arr_f32(theta[L - 1], (size_t)lm * 2 * lm * 2 * lm);
    fan = kin + a.C;
    for (int k = 0; k < nlat; ++k) {
      r.arr_f32(Wlat[L - 1][k], (size_t)a.lat[k] * fan);
      fan = a.lat[k];
    }
  }
  std::vector<std::vector<float>> Wedge(ned + 1);
  fan = a.lat.back();
  for (int k = 0; k <= ned; ++k) {
    int w = (k < ned) ? a.edge[k] : 1;
    r.arr_f32(Wedge[k], (size_t)w * fan);
    fan = w;
  }
  std::vector<double> sigma, mu;
  r.arr_f64(sigma, a.ns);
  r.arr_f64(mu, a.ns);
  if (!r.ok || r.off != bytes) return fail(c, ALLEGRO_E_INVALID, "weights: size mismatch (%zu of %zu bytes)", r.off, bytes);

  // device copies of every linear map
  allegro_status s;
  c->tb.resize(n2);
  fan = a.K0in();
  for (int k = 0; k < n2; ++k) {
    if ((s = upload_lin(c, Wtb[k], a.tb[k], fan, c->tb[k])) != ALLEGRO_OK) return s;
    fan = a.tb[k];
  }
  std::vector<float> W01((size_t)2 * nw * a.tb.back());
  memcpy(W01.data(), Wemb.data(), Wemb.size() * 4);
  memcpy(W01.data() + Wemb.size(), Wenv[0].data(), Wenv[0].size() * 4);
  if ((s = upload_lin(c, W01, 2 * nw, a.tb.back(), c->w01)) != ALLEGRO_OK) return s;
  if (a.nl >= 2 && (s = upload_lin(c, Wenv[1], nw, a.lat.back(), c->env2)) != ALLEGRO_OK) return s;
  if (a.nl >= 3 && (s = upload_lin(c, Wenv[2], nw, a.lat.back(), c->env3)) != ALLEGRO_OK) return s;
  c->lat.assign(a.nl, std::vector<Lin>(nlat));
  for (int L = 1; L <= a.nl; ++L) {
    fan = a.Klat(L - 1) + a.C;
    for (int k = 0; k < nlat; ++k) {
      if ((s = upload_lin(c, Wlat[L - 1][k], a.lat[k], fan, c->lat[L - 1][k])) != ALLEGRO_OK) return s;
      fan = a.lat[k];
    }
  }
  // K-concatenated adjoint maps of x^0 (layer 1: [W_emb ; W_env1] with the latent layer 1_0)
  // and of x^1 (layer 2: W_env2 with the latent layer 2_0)
  for (int L = 1; L <= a.nl; ++L) {
    const std::vector<float>& We = (L == 1) ? W01 : Wenv[L - 1];
    const int K1 = (L == 1) ? 2 * nw : nw;
    const int Nx = a.Klat(L - 1), K2 = a.lat[0], fanl = a.Klat(L - 1) + a.C;
    if (K1 % 64 != 0) continue;
    const int K = K1 + K2, ld = pad8(K);
    std::vector<bf16> hb((size_t)Nx * ld, __float2bfloat16_rn(0.0f));
    for (int n = 0; n < Nx; ++n) {
      for (int k = 0; k < K1; ++k) hb[(size_t)n * ld + k] = __float2bfloat16_rn(We[(size_t)k * Nx + n]);
      for (int k = 0; k < K2; ++k)
        hb[(size_t)n * ld + K1 + k] = __float2bfloat16_rn(Wlat[L - 1][0][(size_t)k * fanl + n]);
    }
    CUDA_TRY(c, cudaMalloc(&c->headB[L - 1], hb.size() * 2));
    c->weight_allocs.push_back(c->headB[L - 1]);
    CUDA_TRY(c, cudaMemcpy(c->headB[L - 1], hb.data(), hb.size() * 2, cudaMemcpyHostToDevice));
    c->headK1[L - 1] = K1; c->headK[L - 1] = K; c->headLd[L - 1] = ld;
    if (c->prec == ALLEGRO_PREC_FP8) {
      // E4M3 copy: float32 rows uploaded to a temporary buffer and quantised there
      std::vector<float> hf((size_t)Nx * K);
      double amax = 0.0;
      for (int n = 0; n < Nx; ++n) {
        for (int k = 0; k < K1; ++k) hf[(size_t)n * K + k] = We[(size_t)k * Nx + n];
        for (int k = 0; k < K2; ++k) hf[(size_t)n * K + K1 + k] = Wlat[L - 1][0][(size_t)k * fanl + n];
      }
      for (float x : hf) amax = std::max(amax, (double)fabsf(x));
      c->headS8[L - 1] = e4m3_weight_scale(amax);
      c->headLd8[L - 1] = (K + 15) / 16 * 16;
      float* tmp = nullptr;
      CUDA_TRY(c, cudaMalloc(&tmp, hf.size() * 4));
      CUDA_TRY(c, cudaMemcpy(tmp, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice));
      CUDA_TRY(c, cudaMalloc(&c->headB8[L - 1], (size_t)Nx * c->headLd8[L - 1]));
      c->weight_allocs.push_back(c->headB8[L - 1]);
      fp8_quantize(tmp, Nx, K, K, c->headB8[L - 1], c->headLd8[L - 1], 1.0f / c->headS8[L - 1], 0);
      const cudaError_t e = cudaDeviceSynchronize();
      cudaFree(tmp);
      if (e != cudaSuccess) return fail(c, ALLEGRO_E_CUDA, "FP8 head weights: %s", cudaGetErrorString(e));
    }
  }
  // linear edge-energy MLP folded into one vector: E_ij = v . x  (float64 product)
  std::vector<double> rvec(1, 1.0);
  for (int k = ned; k >= 0; --k) {
    int out = (k < ned) ? a.edge[k] : 1;
    int in = (k > 0) ? a.edge[k - 1] : a.lat.back();
    std::vector<double> nx(in, 0.0);
    for (int o = 0; o < out; ++o)
      for (int i = 0; i < in; ++i) nx[i] += rvec[o] * (double)Wedge[k][(size_t)o * in + i];
    rvec.swap(nx);
  }
  std::vector<float> v(rvec.begin(), rvec.end());
  CUDA_TRY(c, cudaMalloc(&c->d_v, v.size() * 4));
  c->weight_allocs.push_back(c->d_v);
  CUDA_TRY(c, cudaMemcpy(c->d_v, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMalloc(&c->d_sigma, a.ns * 8));
  c->weight_allocs.push_back(c->d_sigma);
  CUDA_TRY(c, cudaMalloc(&c->d_mu, a.ns * 8));
  c->weight_allocs.push_back(c->d_mu);
  CUDA_TRY(c, cudaMemcpy(c->d_sigma, sigma.data(), a.ns * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_mu, mu.data(), a.ns * 8, cudaMemcpyHostToDevice));

  // tensor-product constants
  const int S = a.S();
  memset(&c->tp, 0, sizeof(c->tp));
  c->tp.nu = (float)(1.0 / sqrt(a.ann));
  if (c->generic) {
    // the fused tensor of every layer between its irreps (pseudo-parity features in the
    // middle layers), packed in the generic row kernels' order
    std::vector<std::vector<Irrep>> irs;
    layer_irreps(a.lmax, a.nl, irs);
    for (int L = 0; L <= a.nl; ++L) {
      c->gdim[L] = irreps_dim(irs[L]);
      if (c->gdim[L] > kGenMaxD) return fail(c, ALLEGRO_E_INVALID, "internal: layer %d has %d components", L, c->gdim[L]);
    }
    std::vector<std::vector<double>> Ws(a.nl + 1);
    for (int L = 1; L <= a.nl; ++L) layer_tensor(a.lmax, irs[L - 1], irs[L], theta[L - 1].data(), Ws[L]);
    std::string why;
    if (!gen_pack_values(a.lmax, a.nl, irs, Ws, c->gen_vals, why))
      return fail(c, ALLEGRO_E_INVALID, "internal: %s", why.c_str());
    return ALLEGRO_OK;
  }
  int nin, nout;
  if (a.nl == 2) {
    std::vector<double> W;
    fused_layer_tensor(a.lmax, theta[0].data(), W, nin, nout, false);
    double wmax = 0.0;
    for (double x : W) wmax = std::max(wmax, fabs(x));
    for (int p = 0; p < S; ++p)
      for (int b = 0; b < S; ++b)
        for (int q = 0; q < S; ++q) {
          const double w = W[((size_t)p * S + b) * S + q];
          if (tp_nonzero(p, b, q)) c->tp.W1[(p * S + b) * S + q] = (float)w;
          else if (fabs(w) > 1e-9 * wmax)   // the kernels skip these entries
            return fail(c, ALLEGRO_E_INVALID, "internal: layer-1 tensor entry (%d,%d,%d) outside the coupling pattern",
                        p, b, q);
        }
  }
  {
    std::vector<double> W;
    fused_layer_tensor(a.lmax, theta[a.nl - 1].data(), W, nin, nout, true);
    for (int p = 0; p < S; ++p)
      for (int b = 0; b < S; ++b) {
        double w = W[(size_t)p * S + b];
        if (p == b) c->tp.clast[p] = (float)w;
        else if (fabs(w) > 1e-12) return fail(c, ALLEGRO_E_INVALID, "internal: last-layer tensor not diagonal");
      }
  }
  return ALLEGRO_OK;
}

// ------------------------------------------------------------------------
// chunk workspace
// ------------------------------------------------------------------------
struct WS {
  // activations (act = float or bf16) and float32 buffers, per chunk edge
  std::vector<void*> Ztb; std::vector<int> ld_Ztb;
  void* H[2]; int ld_H;
  void* X[kGenMaxLayers]; int ld_X[kGenMaxLayers];
  void* Xlast; int ld_Xlast;
  std::vector<std::vector<void*>> Zlat; std::vector<int> ld_Zlat;
  void* W01; int ld_W01;     // [w0 | w1] (activation type)
  void* w2; int ld_w2;       // (activation type)
  void* w3;                  // env weights of layer 3 (three-layer models; pitch ld_w2)
  void* D[kGenMaxLayers]; int ld_D[kGenMaxLayers];   // adjoint of the latent MLP input [x | s], activation type
  void* wbar01; int ld_wbar01;
  void* wbar2; int ld_wbar2;
  void* wbar3;               // (pitch ld_wbar2)
  float* xbar; int ld_xbar;
  float* Y; float* Ybar[2]; float* u; float* ubar; float* sig;
  float* G1; float* G2;
  // generic row path: per atom Gamma^L, Q^L, Gammabar^L (L = 1..nl), Qbar scratch
  float* gG[kGenMaxLayers + 1]; float* gQ[kGenMaxLayers + 1]; float* gGb[kGenMaxLayers + 1];
  float* gQb;
};

// Lays the workspace out over `base` (or only measures it when base is null).
size_t layout_ws(const Arch& a, int act_bytes, int64_t Ec, int64_t Ac, uint8_t* base, WS* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const int ntb = (int)a.tb.size(), nlat = (int)a.lat.size();
  int maxw = 0;
  for (int x : a.tb) maxw = std::max(maxw, x);
  for (int x : a.lat) maxw = std::max(maxw, x);
  const int nw = a.n_w(), S = a.S();
  w->Ztb.resize(ntb); w->ld_Ztb.resize(ntb);
  for (int k = 0; k < ntb; ++k) {
    w->ld_Ztb[k] = pad8(a.tb[k]);
    w->Ztb[k] = take((size_t)Ec * w->ld_Ztb[k] * act_bytes);
  }
  w->ld_H = pad8(maxw);
  w->H[0] = take((size_t)Ec * w->ld_H * act_bytes);
  w->H[1] = take((size_t)Ec * w->ld_H * act_bytes);
  for (int L = 0; L < a.nl; ++L) {
    w->ld_X[L] = pad8(a.Klat(L) + a.C);
    w->X[L] = take((size_t)Ec * w->ld_X[L] * act_bytes);
    w->ld_D[L] = w->ld_X[L];
    w->D[L] = take((size_t)Ec * w->ld_D[L] * act_bytes);
  }
  w->ld_Xlast = pad8(a.lat.back());
  w->Xlast = take((size_t)Ec * w->ld_Xlast * act_bytes);
  w->Zlat.assign(a.nl, std::vector<void*>(nlat));
  w->ld_Zlat.resize(nlat);
  for (int k = 0; k < nlat; ++k) w->ld_Zlat[k] = pad8(a.lat[k]);
  for (int L = 0; L < a.nl; ++L)
    for (int k = 0; k < nlat; ++k) w->Zlat[L][k] = take((size_t)Ec * w->ld_Zlat[k] * act_bytes);
  w->ld_W01 = pad8(2 * nw);
  w->W01 = take((size_t)Ec * w->ld_W01 * act_bytes);
  w->ld_w2 = pad8(nw);
  w->w2 = (a.nl >= 2) ? take((size_t)Ec * w->ld_w2 * act_bytes) : nullptr;
  w->w3 = (a.nl >= 3) ? take((size_t)Ec * w->ld_w2 * act_bytes) : nullptr;
  w->ld_wbar01 = pad8(2 * nw);
  w->wbar01 = take((size_t)Ec * w->ld_wbar01 * act_bytes);
  w->ld_wbar2 = pad8(nw);
  w->wbar2 = (a.nl >= 2) ? take((size_t)Ec * w->ld_wbar2 * act_bytes) : nullptr;
  w->wbar3 = (a.nl >= 3) ? take((size_t)Ec * w->ld_wbar2 * act_bytes) : nullptr;
  const bool generic = a.generic;
  for (int L = 0; L <= kGenMaxLayers; ++L) w->gG[L] = w->gQ[L] = w->gGb[L] = nullptr;
  w->gQb = nullptr;
  if (generic) {
    for (int L = 1; L <= a.nl; ++L) {
      w->gG[L] = (float*)take((size_t)Ac * a.C * S * 4);
      w->gQ[L] = (float*)take((size_t)Ac * a.C * S * 4);
      w->gGb[L] = (float*)take((size_t)Ac * a.C * S * 4);
    }
    w->gQb = (float*)take((size_t)Ac * a.C * S * 4);
  }
  w->ld_xbar = pad8(std::max(a.tb.back(), a.lat.back()));
  w->xbar = (float*)take((size_t)Ec * w->ld_xbar * 4);
  w->Y = (float*)take((size_t)Ec * S * 4);
  for (int k = 0; k < 2; ++k) w->Ybar[k] = (float*)take((size_t)Ec * S * 4);
  w->u = (float*)take((size_t)Ec * 4);
  w->ubar = (float*)take((size_t)Ec * 4);
  w->sig = (float*)take((size_t)Ec * 4);
  w->G1 = (float*)take((size_t)Ac * a.C * S * 4);
  w->G2 = (float*)take((size_t)Ac * a.C * S * 4);
  return off + 256;
}

allegro_status ensure_ws(allegro_ctx* c, int64_t Ec, int64_t Ac, WS* w) {
  const int act_bytes = bf16_storage(c) ? 2 : 4;
  if (Ec > c->ws_edges || Ac > c->ws_atoms || !c->ws) {
    int64_t E2 = std::max<int64_t>(Ec, c->ws_edges), A2 = std::max<int64_t>(Ac, c->ws_atoms);
    E2 = std::max<int64_t>((int64_t)(E2 * 1.05) + 64, 256);
    A2 = std::max<int64_t>((int64_t)(A2 * 1.05) + 16, 64);
    size_t bytes = layout_ws(c->arch, act_bytes, E2, A2, nullptr, w);
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_edges = c->ws_atoms = 0;
    CUDA_TRY(c, cudaMalloc(&c->ws, bytes));
    CUDA_TRY(c, cudaMemset(c->ws, 0, bytes));
    c->ws_bytes = bytes;
    c->ws_edges = E2;
    c->ws_atoms = A2;
  }
  layout_ws(c->arch, act_bytes, c->ws_edges, c->ws_atoms,
            reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(c->ws) + 255) & ~uintptr_t(255)), w);
  return ALLEGRO_OK;
}

int64_t ws_bytes_per_edge(const allegro_ctx* c) {
  WS w;
  const int act_bytes = bf16_storage(c) ? 2 : 4;
  size_t b1 = layout_ws(c->arch, act_bytes, 1 << 16, 1, nullptr, &w);
  return (int64_t)(b1 / (1 << 16)) + 1;
}

// ------------------------------------------------------------------------
// input staging
// ------------------------------------------------------------------------
allegro_status stage_atoms(allegro_ctx* c, int64_t n, const double* pos, const int32_t* types) {
  Caps& k = caps_of(c);
  const int64_t need = std::max<int64_t>(n, 1);
  CUDA_TRY(c, grow(c->d_pos, k.pos, 3 * need));
  CUDA_TRY(c, grow(c->d_types, k.types, need));
  CUDA_TRY(c, grow(c->d_species, k.species, need));
  CUDA_TRY(c, grow(c->d_row_ptr, k.row_ptr, need + 1));
  CUDA_TRY(c, grow(c->d_col_ptr, k.col_ptr, need + 1));
  CUDA_TRY(c, grow(c->d_count, k.count, need + 1));
  CUDA_TRY(c, grow(c->d_cell_of, k.cell_of, need));
  CUDA_TRY(c, grow(c->d_wrap, k.wrap, 3 * need));
  CUDA_TRY(c, grow(c->d_sorted, k.sorted, need));
  CUDA_TRY(c, grow(c->d_pos4, k.pos4, need));
  CUDA_TRY(c, grow(c->d_wraps, k.wraps, need));
  CUDA_TRY(c, grow(c->d_pw, k.pw, 3 * need));
  CUDA_TRY(c, grow(c->d_atom_struct, k.atom_struct, need));
  CUDA_TRY(c, grow(c->d_Eatom, k.Eatom, need));
  CUDA_TRY(c, grow(c->d_F, k.F, 3 * need));
  CUDA_TRY(c, grow(c->d_Wat, k.Wat, 9 * need));
  size_t st = scan_tmp_bytes((int)std::max<int64_t>(need, 4096)) + 4096;
  if (st > c->scan_tmp_cap) {
    if (c->d_scan_tmp) cudaFree(c->d_scan_tmp);
    c->d_scan_tmp = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_scan_tmp, st * 2));
    c->scan_tmp_cap = st * 2;
  }
  if (n > 0) {
    cudaMemcpyKind kp = is_device_ptr(pos) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaMemcpyKind kt = is_device_ptr(types) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_pos, pos, (size_t)n * 3 * 8, kp, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_types, types, (size_t)n * 4, kt, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    map_types_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->d_types, c->d_pos, (int)n, c->d_map,
                                                                         c->nmap, c->d_species, c->d_err);
    CUDA_TRY(c, cudaGetLastError());
  } else {
    CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  }
  return ALLEGRO_OK;
}

allegro_status ensure_structs(allegro_ctx* c, int64_t nstruct) {
  Caps& k = caps_of(c);
  int64_t need = std::max<int64_t>(nstruct, 1);
  CUDA_TRY(c, grow(c->d_offs, k.offs, need + 1));
  CUDA_TRY(c, grow(c->d_cells, k.cells, 9 * need));
  CUDA_TRY(c, grow(c->d_pbc, k.pbc, 3 * need));
  CUDA_TRY(c, grow(c->d_nimg, k.nimg, 3 * need));
  CUDA_TRY(c, grow(c->d_Eout, k.Eout, need));
  CUDA_TRY(c, grow(c->d_Wout, k.Wout, 9 * need));
  return ALLEGRO_OK;
}

allegro_status ensure_edges(allegro_ctx* c, int64_t E) {
  if (c->fixed && c->edge_cap > 0 && E > c->edge_cap)
    return fail(c, ALLEGRO_E_CAPACITY, "neighbour list needs %lld edges, capacity is %lld", (long long)E,
                (long long)c->edge_cap);
  if (E > 2000000000LL) return fail(c, ALLEGRO_E_CAPACITY, "%lld edges exceed the int32 edge index", (long long)E);
  Caps& k = caps_of(c);
  int64_t need = std::max<int64_t>(std::max<int64_t>(E, c->fixed ? c->edge_cap : 0), 1);
  CUDA_TRY(c, grow(c->d_ej, k.ej, need));
  CUDA_TRY(c, grow(c->d_ei, k.ei, need));
  CUDA_TRY(c, grow(c->d_eS, k.eS, 3 * need));
  CUDA_TRY(c, grow(c->d_ed, k.ed, 3 * need));
  CUDA_TRY(c, grow(c->d_col_edge, k.col_edge, need));
  CUDA_TRY(c, grow(c->d_Ee, k.Ee, need));
  CUDA_TRY(c, grow(c->d_g, k.g, 3 * need));
  return ALLEGRO_OK;
}

allegro_status read_err(allegro_ctx* c, int* out) {
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *out = h;
  return ALLEGRO_OK;
}

// CSC index and host row_ptr copy, shared by both neighbour paths.
allegro_status finish_neighbors(allegro_ctx* c, int n, int64_t E) {
  cudaStream_t st = c->stream;
  CUDA_TRY(c, cudaMemsetAsync(c->d_count, 0, (size_t)(n + 1) * 4, st));
  {
    ProfScope ps(c, "nb_csc", 0.0, (double)E * 16 + (double)n * 16, 6);
    nb_columns(c->d_ej, (int)E, n, c->d_count, st);
    exclusive_scan_i32(c->d_count, c->d_col_ptr, n, nullptr, c->d_scan_tmp, c->scan_tmp_cap, st);
    CUDA_TRY(c, cudaMemsetAsync(c->d_count, 0, (size_t)(n + 1) * 4, st));
    nb_fill_columns(c->d_ej, (int)E, c->d_col_ptr, c->d_count, c->d_col_edge, st);
    nb_sort_columns(c->d_col_ptr, n, c->d_col_edge, st);
  }
  CUDA_TRY(c, cudaGetLastError());
  c->h_row_ptr.resize((size_t)n + 1);
  CUDA_TRY(c, cudaMemcpyAsync(c->h_row_ptr.data(), c->d_row_ptr, (size_t)(n + 1) * 4, cudaMemcpyDeviceToHost, st));
  int err = 0;
  allegro_status s = read_err(c, &err);
  if (s != ALLEGRO_OK) return s;
  if (err & kErrBadInput)
    return fail(c, ALLEGRO_E_INVALID, "a type is outside the species map or a position is not finite");
  if (err & kErrNeighbor) return fail(c, ALLEGRO_E_CUDA, "internal: neighbour fill pass disagreed with its count");
  c->n_atoms = n;
  c->n_centres = n;
  c->n_edges = E;
  c->have_nb = true;
  return ALLEGRO_OK;
}

void widths_of(const double* cell, double w[3]) {
  const double* a = cell;
  const double* b = cell + 3;
  const double* cc = cell + 6;
  auto cross = [](const double* x, const double* y, double* o) {
    o[0] = x[1] * y[2] - x[2] * y[1];
    o[1] = x[2] * y[0] - x[0] * y[2];
    o[2] = x[0] * y[1] - x[1] * y[0];
  };
  double bc[3], ca[3], ab[3];
  cross(b, cc, bc); cross(cc, a, ca); cross(a, b, ab);
  double vol = fabs(a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]);
  auto nrm = [](const double* x) { return sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]); };
  w[0] = vol / nrm(bc); w[1] = vol / nrm(ca); w[2] = vol / nrm(ab);
}

bool invert3(const double* m, double* inv) {
  double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
               m[2] * (m[3] * m[7] - m[4] * m[6]);
  if (!(fabs(det) > 0) || !std::isfinite(det)) return false;
  double id = 1.0 / det;
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

// Interned profiling labels: the returned pointer stays valid for the life of
// the process (a deque never moves its elements), from any thread.
static const char* intern_label(const std::string& n) {
  static std::mutex mu;
  static std::deque<std::string> names;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& x : names)
    if (x == n) return x.c_str();
  names.push_back(n);
  return names.back().c_str();
}

// Stable profiling label of a GEMM: which linear map, forward or transposed.
const char* gemm_label(allegro_ctx* c, const Lin* W, bool trans, int epi) {
  std::string n;
  for (size_t k = 0; k < c->tb.size(); ++k)
    if (W == &c->tb[k]) n = "two_body." + std::to_string(k);
  if (W == &c->w01) n = "embed_env1";
  if (W == &c->env2) n = "env2";
  if (W == &c->env3) n = "env3";
  for (size_t L = 0; L < c->lat.size(); ++L)
    for (size_t k = 0; k < c->lat[L].size(); ++k)
      if (W == &c->lat[L][k]) n = "latent." + std::to_string(L + 1) + "." + std::to_string(k);
  const char* en[] = {"silu", "f32", "dsilu", "head", "last", "linear"};
  n = std::string(c->prec == ALLEGRO_PREC_BF16 ? "gemm_tc/"
                  : (c->prec == ALLEGRO_PREC_TF32 ? "gemm_tf32/"
                                                  : (c->prec == ALLEGRO_PREC_FP8 ? "gemm_fp8/" : "gemm_simt/"))) +
      n + (trans ? "^T" : "") + ":" +
      en[epi];
  return intern_label(n);
}

template <typename T>
allegro_status gemm(allegro_ctx* c, GemmArgs g) {
  if (c->prec == ALLEGRO_PREC_BF16) {
    std::string why;
    if (!gemm_tc_bf16(g, c->stream, c->d_err, &why)) return fail(c, ALLEGRO_E_CUDA, "tcgen05 GEMM: %s", why.c_str());
  } else if (c->prec == ALLEGRO_PREC_TF32) {
    std::string why;
    if (!gemm_tc_tf32(g, c->stream, c->d_err, &why)) return fail(c, ALLEGRO_E_CUDA, "tcgen05 TF32 GEMM: %s", why.c_str());
  } else if (c->prec == ALLEGRO_PREC_FP8) {
    std::string why;
    if (!gemm_tc_fp8(g, c->stream, c->d_err, &why)) return fail(c, ALLEGRO_E_CUDA, "tcgen05 FP8 GEMM: %s", why.c_str());
  } else {
    gemm_simt_f32(g, c->stream);
  }
  return ALLEGRO_OK;
}

// Kind of a pair of consecutive layers the fused pair kernel takes (bit of
// Tune::chain_mask): 0 two-body SiLU pair, 1 latent SiLU pair, 2 latent SiLU +
// last layer, 3 head + 256-wide SiLU adjoint, 4 head + narrower SiLU adjoint,
// 5 SiLU adjoint + linear tail.
int pair_kind(const GemmArgs& g1, const GemmArgs& g2) {
  if (g1.epi == EPI_FWD_SILU && g2.epi == EPI_FWD_SILU) return g1.N < 256 ? 0 : 1;
  if (g1.epi == EPI_FWD_SILU && g2.epi == EPI_LAST) return 2;
  if (g1.epi == EPI_HEAD && g2.epi == EPI_BWD_SILU) return g2.N >= 256 ? 3 : 4;
  return 5;
}

// ------------------------------------------------------------------------
// model evaluation of one chunk of whole rows
// ------------------------------------------------------------------------
template <typename T>
allegro_status run_chunk(allegro_ctx* c, const WS& w, int a0, int a1, int e0, int e1, bool backward) {
  const Arch& a = c->arch;
  cudaStream_t st = c->stream;
  const int Ec = e1 - e0, Ac = a1 - a0;
  if (Ec <= 0) return ALLEGRO_OK;
  const int ntb = (int)a.tb.size(), nlat = (int)a.lat.size(), nl = a.nl, nw = a.n_w();
  allegro_status s;
  const double act = sizeof(T);
  auto mk = [&](const void* A, int lda, int K, const Lin& W, bool trans, int epi, void* out, int ldo, int N,
                void* pre = nullptr, int ldp = 0, const float* rowscale = nullptr, const void* add = nullptr,
                int ld_add = 0, float* ubar = nullptr, float* Eout = nullptr) {
    GemmArgs g;
    g.M = Ec; g.N = N; g.K = K; g.A = A; g.lda = lda; g.W = &W; g.trans = trans; g.epi = epi;
    g.out = out; g.ldo = ldo; g.pre = pre; g.ldp = ldp; g.rowscale = rowscale; g.add = add; g.ld_add = ld_add;
    g.ubar = ubar; g.Eout = Eout; g.v = c->d_v; g.rowsig = w.sig;
    g.epq = c->tune.epq_wide;
    return g;
  };
  auto gbytes = [&](const GemmArgs& g, bool count_in, bool count_out) {
    const double outb = (g.epi == EPI_F32) ? 4.0 : act;   // EPI_LINEAR / SiLU modes: activation type
    return (double)Ec * ((count_in ? g.K * act : 0.0) + (count_out ? g.N * outb : 0.0) + (g.pre ? g.N * act : 0.0) +
                         (g.add ? g.N * (g.epi == EPI_HEAD ? act : 4.0) : 0.0) + (g.rowscale ? 4.0 : 0.0)) +
           (double)g.N * g.K * act;
  };
  auto run1 = [&](const GemmArgs& g) {
    ProfScope ps(c, gemm_label(c, g.W, g.trans, g.epi), 2.0 * Ec * (double)g.N * g.K, gbytes(g, true, true));
    return gemm<T>(c, g);
  };
  // Two consecutive layers: one fused kernel when the shapes allow (BF16 path), else two GEMMs.
  auto run2 = [&](const GemmArgs& g1, const GemmArgs& g2) -> allegro_status {
    // Pairs the pipelined chain kernel takes: SiLU -> SiLU and SiLU -> last
    // layer forward, adjoint head -> SiLU adjoint, SiLU adjoint -> linear.  The
    // other pairs run as separate kernels (measured faster).
    const bool want_chain = (g1.epi == EPI_FWD_SILU && (g2.epi == EPI_FWD_SILU || g2.epi == EPI_LAST)) ||
                            (g1.epi == EPI_HEAD && g2.epi == EPI_BWD_SILU) ||
                            (g1.epi == EPI_BWD_SILU && g2.epi == EPI_LINEAR && g2.N <= 256);
    if (c->prec == ALLEGRO_PREC_BF16 && want_chain && (c->tune.chain_mask >> pair_kind(g1, g2) & 1)) {
      std::string why;
      const std::string l2 = gemm_label(c, g2.W, g2.trans, g2.epi);
      const char* label = intern_label(std::string(gemm_label(c, g1.W, g1.trans, g1.epi)) + "+" +
                                       l2.substr(l2.find('/') + 1));
      bool launched;
      {
        ProfScope ps(c, label, 2.0 * Ec * ((double)g1.N * g1.K + (double)g2.N * g2.K),
                     gbytes(g1, true, g1.epi == EPI_BWD_SILU) + gbytes(g2, false, true));
        launched = gemm_chain_bf16(g1, g2, c->stream, c->d_err, &why);
      }
      if (launched) return ALLEGRO_OK;
      if (!why.empty()) return fail(c, ALLEGRO_E_CUDA, "tcgen05 chain GEMM: %s", why.c_str());
    }
    allegro_status r = run1(g1);
    if (r != ALLEGRO_OK) return r;
    GemmArgs g2b = g2;              // separate kernels: layer 2 reads layer 1's output from HBM
    g2b.A = g1.out;
    g2b.lda = g1.ldo;
    return run1(g2b);
  };
  auto G = [&](const void* A, int lda, int K, const Lin& W, bool trans, int epi, void* out, int ldo, int N,
               void* pre = nullptr, int ldp = 0, const float* rowscale = nullptr, const void* add = nullptr,
               int ld_add = 0, float* ubar = nullptr, float* Eout = nullptr) {
    return run1(mk(A, lda, K, W, trans, epi, out, ldo, N, pre, ldp, rowscale, add, ld_add, ubar, Eout));
  };
  RowIO io;
  io.a0 = a0; io.na = Ac; io.e0 = e0; io.row_ptr = c->d_row_ptr; io.C = a.C;
  io.Y = w.Y; io.W01 = w.W01; io.ld01 = w.ld_W01; io.w2 = w.w2; io.ld2 = w.ld_w2; io.G1 = w.G1; io.G2 = w.G2;

  const int S = a.S(), C = a.C;
  // BF16 path: adjoint heads and the edge energy live in the tcgen05 GEMM
  // epilogues, which take whole rows of at most 256 columns; wider MLPs (the
  // paper's 1024-wide production model) run them as the separate elementwise
  // kernels of the float32 paths, with the K-concatenated head GEMMs writing
  // a float32 xbar
  const bool bf16 = (c->prec == ALLEGRO_PREC_BF16);
  const bool fused = bf16 && a.tb.back() <= 256 && a.lat.back() <= 256;
  // algorithmic bytes of the row kernels (per edge, per atom), float32 features
  auto row_scope = [&](const char* name, double per_edge, double per_atom) {
    return ProfScope(c, name, 0.0, (double)Ec * per_edge + (double)Ac * per_atom);
  };
  // ---- forward ----
  // geometry, basis and the first two-body layer in one kernel (its output in H[1], or in X[0]
  // scaled by u when it is the two-body MLP's only layer)
  const bool tb_single = (ntb == 1);
  {
    ProfScope ps(c, "geom_fwd", 2.0 * Ec * a.tb[0] * (a.nb + 2),
                 (double)Ec * (24 + 8 + 8 + S * 4 + 4 + 4 + 2.0 * a.tb[0] * act));
    edge_geom_fwd<T>(Ec, e0, c->d_ed, c->d_ei, c->d_ej, c->d_species, a, w.Y, w.u, c->d_sigma, w.sig,
                     c->tb[0].f32T, c->tb[0].ldT, (T*)w.Ztb[0], w.ld_Ztb[0],
                     (T*)(tb_single ? w.X[0] : w.H[1]), tb_single ? w.ld_X[0] : w.ld_H, tb_single, st);
  }
  const void* in = w.H[1];
  int ld_in = w.ld_H, K = a.tb[0];
  // forward MLP layers [k0, k1) of `layers`: layer k writes pre Z[k], activation to H (or to `last_out`)
  // layers [k0, nlay) of `layers`; layer k writes its activation to H[(k - k0) & 1] (or to `last_out`)
  auto fwd_mlp = [&](const std::vector<Lin>& layers, const std::vector<void*>& Z, const std::vector<int>& ldZ,
                     int k0, int nlay, const void*& src, int& ld_src, int& Kin, void* last_out,
                     int ld_last) -> allegro_status {
    int k = k0;
    while (k < nlay) {
      const bool last = (k == nlay - 1);
      void* out = last ? last_out : w.H[(k - k0) & 1];
      int ldo = last ? ld_last : w.ld_H;
      GemmArgs g1 = mk(src, ld_src, Kin, layers[k], false, EPI_FWD_SILU, out, ldo, layers[k].N, Z[k], ldZ[k],
                       last ? w.u : nullptr);
      if (k + 1 < nlay && k + 1 == nlay - 1 && k >= 0) {
        // chain the last two layers (the intermediate activation stays on chip)
        GemmArgs g2 = mk(nullptr, 0, layers[k].N, layers[k + 1], false, EPI_FWD_SILU, last_out, ld_last,
                         layers[k + 1].N, Z[k + 1], ldZ[k + 1], w.u);
        g1.rowscale = nullptr;
        g1.out = w.H[(k - k0) & 1]; g1.ldo = w.ld_H;
        allegro_status r = run2(g1, g2);
        if (r != ALLEGRO_OK) return r;
        src = last_out; ld_src = ld_last; Kin = layers[k + 1].N;
        return ALLEGRO_OK;
      }
      allegro_status r = run1(g1);
      if (r != ALLEGRO_OK) return r;
      src = out; ld_src = ldo; Kin = layers[k].N;
      ++k;
    }
    return ALLEGRO_OK;
  };
  if (ntb > 1 && (s = fwd_mlp(c->tb, w.Ztb, w.ld_Ztb, 1, ntb, in, ld_in, K, w.X[0], w.ld_X[0])) != ALLEGRO_OK)
    return s;
  if ((s = G(w.X[0], w.ld_X[0], a.tb.back(), c->w01, false, EPI_LINEAR, w.W01, w.ld_W01, 2 * nw)) != ALLEGRO_OK)
    return s;
  for (int L = 1; L <= nl; ++L) {
    io.xs = w.X[L - 1]; io.ldxs = w.ld_X[L - 1]; io.xs_off = a.Klat(L - 1);
    {
      const double pe = (L < nl) ? (2.0 * nw * act + S * 4 + C * act)
                                 : ((L == 1 ? 2.0 : 3.0) * nw * act + S * 4 + C * act);
      const double pa = (L < nl) ? C * S * 4.0 : (L == 1 ? 1.0 : 2.0) * C * S * 4.0;
      auto ps = row_scope(L < nl ? "row_fwd_mid" : "row_fwd_last", pe, pa);
      row_fwd<T>(L, nl, a.lmax, io, c->tp, st);
    }
    in = w.X[L - 1]; ld_in = w.ld_X[L - 1]; K = a.Klat(L - 1) + a.C;
    if (fused && L == nl) {
      // last latent MLP; its final layer carries the folded edge energy and the start of the adjoint
      if (nlat >= 2) {
        if ((s = fwd_mlp(c->lat[L - 1], w.Zlat[L - 1], w.ld_Zlat, 0, nlat - 2, in, ld_in, K, nullptr, 0)) !=
            ALLEGRO_OK)
          return s;
        GemmArgs g1 = mk(in, ld_in, K, c->lat[L - 1][nlat - 2], false, EPI_FWD_SILU, w.H[1], w.ld_H,
                         a.lat[nlat - 2], w.Zlat[L - 1][nlat - 2], w.ld_Zlat[nlat - 2]);
        GemmArgs g2 = mk(nullptr, 0, a.lat[nlat - 2], c->lat[L - 1][nlat - 1], false, EPI_LAST, w.H[0], w.ld_H,
                         a.lat[nlat - 1], nullptr, 0, w.u, nullptr, 0, w.ubar, c->d_Ee + e0);
        if ((s = run2(g1, g2)) != ALLEGRO_OK) return s;
      } else if ((s = G(in, ld_in, K, c->lat[L - 1][0], false, EPI_LAST, w.H[0], w.ld_H, a.lat[0], nullptr, 0, w.u,
                        nullptr, 0, w.ubar, c->d_Ee + e0)) != ALLEGRO_OK) {
        return s;
      }
    } else {
      void* dst = (L < nl) ? w.X[L] : w.Xlast;
      const int ld_dst = (L < nl) ? w.ld_X[L] : w.ld_Xlast;
      if ((s = fwd_mlp(c->lat[L - 1], w.Zlat[L - 1], w.ld_Zlat, 0, nlat, in, ld_in, K, dst, ld_dst)) != ALLEGRO_OK)
        return s;
    }
    if (L < nl) {
      if ((s = G(w.X[L], w.ld_X[L], a.lat.back(), c->env2, false, EPI_LINEAR, w.w2, w.ld_w2, nw)) != ALLEGRO_OK)
        return s;
    }
  }
  if (!fused) {
    ProfScope ps(c, "edge_energy", 0.0, (double)Ec * (a.lat.back() * act + 4));
    edge_energy<T>(Ec, a.lat.back(), (const T*)w.Xlast, w.ld_Xlast, c->d_v, c->d_Ee + e0, st);
  }
  if (!backward) return ALLEGRO_OK;

  // ---- adjoint ----
  // latent MLP of the last layer: xbar = sigma_{Z_i} v (fused into EPI_LAST on the BF16 path)
  if (!fused) {
    ProfScope ps(c, "head_bwd", 0.0, (double)Ec * (a.lat.back() * 2 * act + 16));
    mlp_head_bwd<T>(Ec, a.lat.back(), nullptr, 0, c->d_v, c->d_ei, c->d_species, c->d_sigma, e0,
                    (const T*)w.Zlat[nl - 1][nlat - 1], w.ld_Zlat[nlat - 1], w.u, w.ubar, true, (T*)w.H[0], w.ld_H,
                    st);
  }
  // Adjoint of an MLP: transposed GEMMs down to the input adjoint (columns [col0, Kin) of the
  // input, written at dst + col0); *zin receives the adjoint of layer 0's pre-activation (the
  // last GEMM's A operand).  `head`, if given, is the GEMM that forms the adjoint of the last
  // layer's pre-activation (into H[0]); it runs paired with the first transposed GEMM.
  auto back_mlp = [&](const std::vector<Lin>& layers, const std::vector<void*>& Z, const std::vector<int>& ldZ,
                      int nlay, void* dst, int ld_dst, int Kin, int epi_dst, int col0, const void** zin,
                      const GemmArgs* head) -> allegro_status {
    int cur = 0;
    int k = nlay - 1;
    if (head && nlay < 2) {
      allegro_status r = run1(*head);
      if (r != ALLEGRO_OK) return r;
      head = nullptr;
    }
    void* dstc = col0 ? (void*)((char*)dst + (size_t)col0 * sizeof(T)) : dst;
    auto last = [&](const void* A, const Lin& W0) {
      GemmArgs g = mk(A, w.ld_H, W0.N, W0, true, epi_dst, dstc, ld_dst, Kin - col0);
      g.b_row0 = col0;
      if (zin) *zin = A;
      return g;
    };
    while (k >= 0) {
      const Lin& W = layers[k];
      allegro_status r;
      if (k >= 1) {
        GemmArgs g1 = mk(w.H[cur], w.ld_H, W.N, W, true, EPI_BWD_SILU, w.H[cur ^ 1], w.ld_H, W.K, Z[k - 1], ldZ[k - 1]);
        const Lin& W2 = layers[k - 1];
        if (head) {
          // the head's product stays on chip as the A operand of this layer's GEMM
          if ((r = run2(*head, g1)) != ALLEGRO_OK) return r;
          head = nullptr;
          cur ^= 1;
          --k;
          continue;
        }
        if (k - 1 == 0) {
          // layer 1's product (written to HBM for the head GEMM of the layer below) stays on chip
          // as the A operand of layer 0's GEMM
          if ((r = run2(g1, last(w.H[cur ^ 1], W2))) != ALLEGRO_OK) return r;
        } else {
          GemmArgs g2 = mk(nullptr, 0, W2.N, W2, true, EPI_BWD_SILU, w.H[cur], w.ld_H, W2.K, Z[k - 2], ldZ[k - 2]);
          if ((r = run2(g1, g2)) != ALLEGRO_OK) return r;
        }
        k -= 2;
        continue;
      }
      if ((r = run1(last(w.H[cur], W))) != ALLEGRO_OK) return r;
      --k;
    }
    return ALLEGRO_OK;
  };
  // BF16 path with a K-concatenated head map: the latent MLP adjoint writes only the s columns of
  // D; the head GEMM forms the x columns from [wbar | zbar] directly
  auto kcat = [&](int L) { return bf16 && c->headB[L - 1] != nullptr; };
  if (bf16 && !fused && (!kcat(1) || (nl == 2 && !kcat(2))))
    return fail(c, ALLEGRO_E_INVALID, "BF16 path with MLPs wider than 256 needs 64-aligned env-weight widths");
  // D (the latent inputs' adjoint) is stored in the activation type: EPI_LINEAR
  const void* zlat[2] = {nullptr, nullptr};
  if ((s = back_mlp(c->lat[nl - 1], w.Zlat[nl - 1], w.ld_Zlat, nlat, w.D[nl - 1], w.ld_D[nl - 1],
                    a.Klat(nl - 1) + a.C, EPI_LINEAR, kcat(nl) ? a.Klat(nl - 1) : 0, &zlat[nl - 1], nullptr)) !=
      ALLEGRO_OK)
    return s;
  io.wbar01 = w.wbar01; io.ld_wbar01 = w.ld_wbar01; io.wbar2 = w.wbar2; io.ld_wbar2 = w.ld_wbar2;
  for (int k = 0; k < 2; ++k) io.Ybar[k] = w.Ybar[k];
  if (nl == 1) {
    io.sbar1 = (const T*)w.D[0] + a.Klat(0); io.ld_sbar1 = w.ld_D[0];
    auto ps = row_scope("row_bwd_last", 2.0 * nw * act + C * act + S * 4 + 2.0 * nw * act + 2 * S * 4, C * S * 4.0);
    row_bwd<T>(1, 1, a.lmax, io, c->tp, st);
  } else {
    io.sbar2 = (const T*)w.D[1] + a.Klat(1); io.ld_sbar2 = w.ld_D[1];
    {
      auto ps = row_scope("row_bwd_last", 2.0 * nw * act + C * act + S * 4 + nw * act + S * 4, 2.0 * C * S * 4);
      row_bwd<T>(2, 2, a.lmax, io, c->tp, st);
    }
    // xbar^1 = wbar^2 . env2 + D[1][:, :K1], then the adjoint head of x^1 = u silu(z)
    GemmArgs head1;
    const GemmArgs* head1p = nullptr;
    if (kcat(2) && !fused) {
      // wide MLPs: xbar^1 in float32 from the K-concatenated GEMM, the head below
      head1 = mk(w.wbar2, w.ld_wbar2, c->headK[1], c->env2, true, EPI_F32, w.xbar, w.ld_xbar, a.lat.back());
      head1.A2 = zlat[1]; head1.lda2 = w.ld_H; head1.K1 = c->headK1[1];
      head1.Bover = c->headB[1]; head1.ldb_over = c->headLd[1];
      if ((s = run1(head1)) != ALLEGRO_OK) return s;
    } else if (kcat(2)) {
      head1 = mk(w.wbar2, w.ld_wbar2, c->headK[1], c->env2, true, EPI_HEAD, w.H[0], w.ld_H, a.lat.back(),
                 w.Zlat[0][nlat - 1], w.ld_Zlat[nlat - 1], w.u, nullptr, 0, w.ubar);
      head1.A2 = zlat[1]; head1.lda2 = w.ld_H; head1.K1 = c->headK1[1];
      head1.Bover = c->headB[1]; head1.ldb_over = c->headLd[1];
      head1p = &head1;   // runs paired with the first GEMM of the latent MLP adjoint below
    } else if (fused) {
      if ((s = G(w.wbar2, w.ld_wbar2, nw, c->env2, true, EPI_HEAD, w.H[0], w.ld_H, a.lat.back(),
                 w.Zlat[0][nlat - 1], w.ld_Zlat[nlat - 1], w.u, w.D[1], w.ld_D[1], w.ubar)) != ALLEGRO_OK)
        return s;
    } else if ((s = G(w.wbar2, w.ld_wbar2, nw, c->env2, true, EPI_F32, w.xbar, w.ld_xbar, a.lat.back(), nullptr,
                      0, nullptr, w.D[1], w.ld_D[1])) != ALLEGRO_OK) {
      return s;
    }
    if (!fused) {
      ProfScope ps(c, "head_bwd", 0.0, (double)Ec * (a.lat.back() * (4 + 2 * act) + 12));
      mlp_head_bwd<T>(Ec, a.lat.back(), w.xbar, w.ld_xbar, nullptr, c->d_ei, c->d_species, c->d_sigma, e0,
                      (const T*)w.Zlat[0][nlat - 1], w.ld_Zlat[nlat - 1], w.u, w.ubar, false, (T*)w.H[0], w.ld_H,
                      st);
    }
    if ((s = back_mlp(c->lat[0], w.Zlat[0], w.ld_Zlat, nlat, w.D[0], w.ld_D[0], a.Klat(0) + a.C, EPI_LINEAR,
                      kcat(1) ? a.Klat(0) : 0, &zlat[0], head1p)) != ALLEGRO_OK)
      return s;
    io.sbar1 = (const T*)w.D[0] + a.Klat(0); io.ld_sbar1 = w.ld_D[0];
    auto ps = row_scope("row_bwd_mid", 2.0 * nw * act + 2.0 * C * act + S * 4 + 2.0 * nw * act + S * 4,
                        2.0 * C * S * 4);
    row_bwd<T>(1, 2, a.lmax, io, c->tp, st);
  }
  // xbar^0 = [wbar^0 | wbar^1] . [W_emb ; W_env1] + D[0][:, :K0], then the head of x^0 = u silu(z)
  GemmArgs head0;
  bool head0_pending = false;
  if (kcat(1) && !fused) {
    // wide MLPs: xbar^0 in float32 from the K-concatenated GEMM, the head below
    head0 = mk(w.wbar01, w.ld_wbar01, c->headK[0], c->w01, true, EPI_F32, w.xbar, w.ld_xbar, a.tb.back());
    head0.A2 = zlat[0]; head0.lda2 = w.ld_H; head0.K1 = c->headK1[0];
    head0.Bover = c->headB[0]; head0.ldb_over = c->headLd[0];
    if ((s = run1(head0)) != ALLEGRO_OK) return s;
  } else if (kcat(1)) {
    head0 = mk(w.wbar01, w.ld_wbar01, c->headK[0], c->w01, true, EPI_HEAD, w.H[0], w.ld_H, a.tb.back(),
               w.Ztb[ntb - 1], w.ld_Ztb[ntb - 1], w.u, nullptr, 0, w.ubar);
    head0.A2 = zlat[0]; head0.lda2 = w.ld_H; head0.K1 = c->headK1[0];
    head0.Bover = c->headB[0]; head0.ldb_over = c->headLd[0];
    if (ntb >= 2) head0_pending = true;   // paired with the last two-body layer's GEMM below
    else if ((s = run1(head0)) != ALLEGRO_OK) return s;
  } else if (fused) {
    if ((s = G(w.wbar01, w.ld_wbar01, 2 * nw, c->w01, true, EPI_HEAD, w.H[0], w.ld_H, a.tb.back(),
               w.Ztb[ntb - 1], w.ld_Ztb[ntb - 1], w.u, w.D[0], w.ld_D[0], w.ubar)) != ALLEGRO_OK)
      return s;
  } else if ((s = G(w.wbar01, w.ld_wbar01, 2 * nw, c->w01, true, EPI_F32, w.xbar, w.ld_xbar, a.tb.back(), nullptr,
                    0, nullptr, w.D[0], w.ld_D[0])) != ALLEGRO_OK) {
    return s;
  }
  if (!fused) {
    ProfScope ps(c, "head_bwd", 0.0, (double)Ec * (a.tb.back() * (4 + 2 * act) + 12));
    mlp_head_bwd<T>(Ec, a.tb.back(), w.xbar, w.ld_xbar, nullptr, c->d_ei, c->d_species, c->d_sigma, e0,
                    (const T*)w.Ztb[ntb - 1], w.ld_Ztb[ntb - 1], w.u, w.ubar, false, (T*)w.H[0], w.ld_H, st);
  }
  // two-body MLP adjoint down to zbar0; the first layer's transposed product is folded into geom_bwd
  int cur0 = 0;
  for (int k = ntb - 1; k >= 1; --k) {
    const Lin& W = c->tb[k];
    GemmArgs g = mk(w.H[cur0], w.ld_H, W.N, W, true, EPI_BWD_SILU, w.H[cur0 ^ 1], w.ld_H, W.K, w.Ztb[k - 1],
                    w.ld_Ztb[k - 1]);
    if (head0_pending) {
      s = run2(head0, g);
      head0_pending = false;
    } else {
      s = run1(g);
    }
    if (s != ALLEGRO_OK) return s;
    cur0 ^= 1;
  }
  {
    ProfScope ps(c, "geom_bwd", 2.0 * Ec * a.tb[0] * a.nb,
                 (double)Ec * (24 + a.tb[0] * act + 4 + 2 * S * 4 + 12));
    YbarParts yb{{w.Ybar[0], w.Ybar[1]}};
    edge_geom_bwd<T>(Ec, e0, c->d_ed, c->d_ei, c->d_ej, c->d_species, a, (const T*)w.H[cur0], w.ld_H, c->tb[0].f32T, c->tb[0].ldT, w.ubar, yb,
                     c->d_g, st);
  }
  return ALLEGRO_OK;
}

// One chunk through the generic row path (three layers, or l_max 3): the
// environment sums and products of row_generic.cu, the MLPs as single GEMMs
// with the heads and the edge energy as elementwise kernels (BF16: the heads'
// K-concatenated GEMMs write a float32 xbar), any number of layers.
template <typename T>
allegro_status run_chunk_gen(allegro_ctx* c, const WS& w, int a0, int a1, int e0, int e1, bool backward) {
  const Arch& a = c->arch;
  cudaStream_t st = c->stream;
  const int Ec = e1 - e0, Ac = a1 - a0;
  if (Ec <= 0) return ALLEGRO_OK;
  const int ntb = (int)a.tb.size(), nlat = (int)a.lat.size(), nl = a.nl, nw = a.n_w(), S = a.S();
  const bool bf16 = bf16_storage(c);
  const bool fp8 = (c->prec == ALLEGRO_PREC_FP8);
  allegro_status s;
  const double act = sizeof(T);
  // FP8: per-tensor amax slots.  Every kernel that writes a whole activation array an
  // E4M3 GEMM reads takes a fresh slot for it; a GEMM reads the latest slot of its
  // operand arrays (the s columns written into [x | s] join the slot of x).
  const void* slot_buf[kAmaxSlots];
  int nslot = 0;
  bool slots_exhausted = false;   // reported after the chunk (the kernels ran without a record)
  auto fresh = [&](const void* b) -> unsigned* {
    if (!fp8) return nullptr;
    if (nslot >= kAmaxSlots) {
      slots_exhausted = true;
      return nullptr;
    }
    slot_buf[nslot] = b;
    return c->d_amax + nslot++;
  };
  auto slot_of = [&](const void* b) -> unsigned* {
    if (!fp8 || !b) return nullptr;
    for (int k = nslot - 1; k >= 0; --k)
      if (slot_buf[k] == b) return c->d_amax + k;
    return nullptr;
  };
  if (fp8) CUDA_TRY(c, cudaMemsetAsync(c->d_amax, 0, kAmaxSlots * sizeof(unsigned), st));
  auto mk = [&](const void* A, int lda, int K, const Lin& W, bool trans, int epi, void* out, int ldo, int N,
                void* pre = nullptr, int ldp = 0, const float* rowscale = nullptr, const void* add = nullptr,
                int ld_add = 0) {
    GemmArgs g;
    g.M = Ec; g.N = N; g.K = K; g.A = A; g.lda = lda; g.W = &W; g.trans = trans; g.epi = epi;
    g.out = out; g.ldo = ldo; g.pre = pre; g.ldp = ldp; g.rowscale = rowscale; g.add = add; g.ld_add = ld_add;
    g.v = c->d_v; g.rowsig = w.sig; g.epq = c->tune.epq_wide;
    return g;
  };
  auto run1 = [&](GemmArgs g) {
    if (fp8) {
      g.amax_a = slot_of(g.A);
      g.amax_a2 = slot_of(g.A2);
      if (g.epi == EPI_FWD_SILU || g.epi == EPI_BWD_SILU) {
        g.amax_out = fresh(g.out);
        if (!g.amax_out) return fail(c, ALLEGRO_E_INVALID, "FP8: more than %d activation arrays in a chunk", kAmaxSlots);
      }
    }
    const double outb = (g.epi == EPI_F32) ? 4.0 : act;
    ProfScope ps(c, gemm_label(c, g.W, g.trans, g.epi), 2.0 * Ec * (double)g.N * g.K,
                 (double)Ec * (g.K * act + g.N * outb + (g.pre ? g.N * act : 0.0)) + (double)g.N * g.K * act);
    return gemm<T>(c, g);
  };
  // forward MLP layers [k0, nlay): SiLU, pre-activations kept, the last layer times u into last_out
  auto fwd_mlp = [&](const std::vector<Lin>& layers, const std::vector<void*>& Z, const std::vector<int>& ldZ,
                     int k0, int nlay, const void* src, int ld_src, int Kin, void* last_out,
                     int ld_last) -> allegro_status {
    for (int k = k0; k < nlay; ++k) {
      const bool last = (k == nlay - 1);
      void* out = last ? last_out : w.H[(k - k0) & 1];
      const int ldo = last ? ld_last : w.ld_H;
      allegro_status r = run1(mk(src, ld_src, Kin, layers[k], false, EPI_FWD_SILU, out, ldo, layers[k].N, Z[k],
                                 ldZ[k], last ? w.u : nullptr));
      if (r != ALLEGRO_OK) return r;
      src = out; ld_src = ldo; Kin = layers[k].N;
    }
    return ALLEGRO_OK;
  };
  // adjoint of an MLP from zbar of its last layer (in H[0]) to its input's adjoint, columns [col0, Kin)
  auto back_mlp = [&](const std::vector<Lin>& layers, const std::vector<void*>& Z, const std::vector<int>& ldZ,
                      void* dst, int ld_dst, int Kin, int col0, const void** zin) -> allegro_status {
    int cur = 0;
    for (int k = (int)layers.size() - 1; k >= 0; --k) {
      const Lin& W = layers[k];
      allegro_status r;
      if (k >= 1) {
        r = run1(mk(w.H[cur], w.ld_H, W.N, W, true, EPI_BWD_SILU, w.H[cur ^ 1], w.ld_H, W.K, Z[k - 1], ldZ[k - 1]));
        cur ^= 1;
      } else {
        void* dstc = col0 ? (void*)((char*)dst + (size_t)col0 * sizeof(T)) : dst;
        GemmArgs g = mk(w.H[cur], w.ld_H, W.N, W, true, EPI_LINEAR, dstc, ld_dst, Kin - col0);
        g.b_row0 = col0;
        if (zin) *zin = w.H[cur];
        r = run1(g);
      }
      if (r != ALLEGRO_OK) return r;
    }
    return ALLEGRO_OK;
  };
  const Lin* env[kGenMaxLayers + 1] = {nullptr, &c->w01, &c->env2, &c->env3};
  void* wL[kGenMaxLayers + 1] = {w.W01, w.W01, w.w2, w.w3};
  void* wbL[kGenMaxLayers + 1] = {w.wbar01, w.wbar01, w.wbar2, w.wbar3};
  GenRowIO gio;
  gio.a0 = a0; gio.na = Ac; gio.e0 = e0; gio.C = a.C; gio.S = S; gio.lmax = a.lmax; gio.nl = nl;
  gio.row_ptr = c->d_row_ptr; gio.Y = w.Y; gio.nu = c->tp.nu; gio.Qb = w.gQb;
  gio.Ybar = w.Ybar[0];
  gio.vals = c->gen_vals.data();
  for (int L = 0; L <= nl; ++L) {
    gio.w[L] = wL[L];
    gio.ldw[L] = (L <= 1) ? w.ld_W01 : w.ld_w2;
    gio.wcol[L] = (L == 1) ? nw : 0;
    gio.wbar[L] = wbL[L];
    gio.ldwbar[L] = (L <= 1) ? w.ld_wbar01 : w.ld_wbar2;
    gio.wbcol[L] = (L == 1) ? nw : 0;
    gio.dim[L] = c->gdim[L];
    if (L >= 1) {
      gio.xs[L] = w.X[L - 1]; gio.ldxs[L] = w.ld_X[L - 1]; gio.xs_off[L] = a.Klat(L - 1);
      gio.sbar[L] = w.D[L - 1]; gio.ldsbar[L] = w.ld_D[L - 1]; gio.sbar_off[L] = a.Klat(L - 1);
      gio.G[L] = w.gG[L]; gio.Q[L] = w.gQ[L]; gio.Gb[L] = w.gGb[L];
    }
  }
  // ---- forward ----
  const bool tb_single = (ntb == 1);
  {
    ProfScope ps(c, "geom_fwd", 2.0 * Ec * a.tb[0] * (a.nb + 2),
                 (double)Ec * (24 + 8 + 8 + S * 4 + 4 + 4 + 2.0 * a.tb[0] * act));
    edge_geom_fwd<T>(Ec, e0, c->d_ed, c->d_ei, c->d_ej, c->d_species, a, w.Y, w.u, c->d_sigma, w.sig,
                     c->tb[0].f32T, c->tb[0].ldT, (T*)w.Ztb[0], w.ld_Ztb[0],
                     (T*)(tb_single ? w.X[0] : w.H[1]), tb_single ? w.ld_X[0] : w.ld_H, tb_single, st,
                     fresh(tb_single ? w.X[0] : w.H[1]));
  }
  if (ntb > 1 && (s = fwd_mlp(c->tb, w.Ztb, w.ld_Ztb, 1, ntb, w.H[1], w.ld_H, a.tb[0], w.X[0], w.ld_X[0])) != ALLEGRO_OK)
    return s;
  if ((s = run1(mk(w.X[0], w.ld_X[0], a.tb.back(), c->w01, false, EPI_LINEAR, w.W01, w.ld_W01, 2 * nw))) != ALLEGRO_OK)
    return s;
  for (int L = 1; L <= nl; ++L) {
    if (L >= 2 &&
        (s = run1(mk(w.X[L - 1], w.ld_X[L - 1], a.lat.back(), *env[L], false, EPI_LINEAR, wL[L], w.ld_w2, nw))) !=
            ALLEGRO_OK)
      return s;
    {
      ProfScope ps(c, "row_gen_fwd", 0.0, (double)Ec * (2.0 * nw * act + S * 4 + a.C * act) + (double)Ac * a.C * S * 8.0, 3);
      gio.amax_s = slot_of(w.X[L - 1]);
      gen_row_fwd<T>(gio, L, st);
    }
    void* dst = (L < nl) ? w.X[L] : w.Xlast;
    const int ld_dst = (L < nl) ? w.ld_X[L] : w.ld_Xlast;
    if ((s = fwd_mlp(c->lat[L - 1], w.Zlat[L - 1], w.ld_Zlat, 0, nlat, w.X[L - 1], w.ld_X[L - 1],
                     a.Klat(L - 1) + a.C, dst, ld_dst)) != ALLEGRO_OK)
      return s;
  }
  {
    ProfScope ps(c, "edge_energy", 0.0, (double)Ec * (a.lat.back() * act + 4));
    edge_energy<T>(Ec, a.lat.back(), (const T*)w.Xlast, w.ld_Xlast, c->d_v, c->d_Ee + e0, st);
  }
  if (slots_exhausted)
    return fail(c, ALLEGRO_E_INVALID, "FP8: more than %d activation arrays in a chunk", kAmaxSlots);
  if (!backward) return ALLEGRO_OK;
  // ---- adjoint ----
  {
    ProfScope ps(c, "head_bwd", 0.0, (double)Ec * (a.lat.back() * 2 * act + 16));
    mlp_head_bwd<T>(Ec, a.lat.back(), nullptr, 0, c->d_v, c->d_ei, c->d_species, c->d_sigma, e0,
                    (const T*)w.Zlat[nl - 1][nlat - 1], w.ld_Zlat[nlat - 1], w.u, w.ubar, true, (T*)w.H[0], w.ld_H,
                    st, fresh(w.H[0]));
  }
  for (int L = nl; L >= 1; --L) {
    const bool kc = bf16 && c->headB[L - 1] != nullptr && (!fp8 || c->headB8[L - 1] != nullptr);
    const void* zlat = nullptr;
    if ((s = back_mlp(c->lat[L - 1], w.Zlat[L - 1], w.ld_Zlat, w.D[L - 1], w.ld_D[L - 1], a.Klat(L - 1) + a.C,
                      kc ? a.Klat(L - 1) : 0, &zlat)) != ALLEGRO_OK)
      return s;
    {
      ProfScope ps(c, "row_gen_bwd", 0.0, (double)Ec * (4.0 * nw * act + 2 * S * 4 + a.C * act) + (double)Ac * a.C * S * 16.0, 3);
      gio.amax_wbar = fresh(wbL[L]);
      gen_row_bwd<T>(gio, L, st);
    }
    // xbar of x^{L-1} = wbar^L . W_env^L (layer 1: [wbar^0 | wbar^1] . [W_emb ; W_env^1]) + its latent-input adjoint
    const int K1 = (L == 1) ? 2 * nw : nw;
    GemmArgs hd;
    if (kc) {
      hd = mk(wbL[L], (L == 1) ? w.ld_wbar01 : w.ld_wbar2, c->headK[L - 1], *env[L], true, EPI_F32, w.xbar,
              w.ld_xbar, a.Klat(L - 1));
      hd.A2 = zlat; hd.lda2 = w.ld_H; hd.K1 = c->headK1[L - 1];
      hd.Bover = c->headB[L - 1]; hd.ldb_over = c->headLd[L - 1];
      hd.Bover8 = c->headB8[L - 1]; hd.ldb_over8 = c->headLd8[L - 1]; hd.sBover8 = c->headS8[L - 1];
    } else if (bf16) {
      // env-weight widths off the 64-column k-blocks: wbar . W_env in float32, the latent input's
      // adjoint (bf16) added by the head kernel below
      hd = mk(wbL[L], (L == 1) ? w.ld_wbar01 : w.ld_wbar2, K1, *env[L], true, EPI_F32, w.xbar, w.ld_xbar,
              a.Klat(L - 1));
    } else {
      hd = mk(wbL[L], (L == 1) ? w.ld_wbar01 : w.ld_wbar2, K1, *env[L], true, EPI_F32, w.xbar, w.ld_xbar,
              a.Klat(L - 1), nullptr, 0, nullptr, w.D[L - 1], w.ld_D[L - 1]);
    }
    if ((s = run1(hd)) != ALLEGRO_OK) return s;
    const void* pre = (L == 1) ? w.Ztb[ntb - 1] : w.Zlat[L - 2][nlat - 1];
    const int ldp = (L == 1) ? w.ld_Ztb[ntb - 1] : w.ld_Zlat[nlat - 1];
    ProfScope ps(c, "head_bwd", 0.0, (double)Ec * (a.Klat(L - 1) * (4 + 2 * act) + 12));
    mlp_head_bwd<T>(Ec, a.Klat(L - 1), w.xbar, w.ld_xbar, nullptr, c->d_ei, c->d_species, c->d_sigma, e0,
                    (const T*)pre, ldp, w.u, w.ubar, false, (T*)w.H[0], w.ld_H, st, fresh(w.H[0]),
                    (bf16 && !kc) ? (const T*)w.D[L - 1] : nullptr, w.ld_D[L - 1]);
  }
  int cur0 = 0;
  for (int k = ntb - 1; k >= 1; --k) {
    const Lin& W = c->tb[k];
    if ((s = run1(mk(w.H[cur0], w.ld_H, W.N, W, true, EPI_BWD_SILU, w.H[cur0 ^ 1], w.ld_H, W.K, w.Ztb[k - 1],
                     w.ld_Ztb[k - 1]))) != ALLEGRO_OK)
      return s;
    cur0 ^= 1;
  }
  {
    ProfScope ps(c, "geom_bwd", 2.0 * Ec * a.tb[0] * a.nb, (double)Ec * (24 + a.tb[0] * act + 4 + S * 4 + 12));
    YbarParts yb{{w.Ybar[0], nullptr}};
    edge_geom_bwd<T>(Ec, e0, c->d_ed, c->d_ei, c->d_ej, c->d_species, a, (const T*)w.H[cur0], w.ld_H,
                     c->tb[0].f32T, c->tb[0].ldT, w.ubar, yb, c->d_g, st);
  }
  if (slots_exhausted)
    return fail(c, ALLEGRO_E_INVALID, "FP8: more than %d activation arrays in a chunk", kAmaxSlots);
  return ALLEGRO_OK;
}

// Chunks of whole rows (each centre's environment sum complete inside one
// chunk), at most `budget` edges each (0: the largest the memory allows).
struct Plan {
  std::vector<int> bounds;
  int64_t maxE = 1, maxA = 1;
};

Plan plan_chunks(allegro_ctx* c, int64_t budget) {
  const int n = (int)c->n_atoms;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    int64_t per = ws_bytes_per_edge(c);
    int64_t cap_bytes = std::min<int64_t>((int64_t)(fr * 0.5) + (int64_t)c->ws_bytes, 48ll << 30);
    budget = std::max<int64_t>(cap_bytes / std::max<int64_t>(per, 1), 1 << 16);
  }
  Plan p;
  p.bounds.push_back(0);
  int a = 0;
  while (a < n) {
    int64_t start = c->h_row_ptr[a];
    // largest b with row_ptr[b] - start <= budget (at least one row)
    int lo = a + 1, hi = n;
    while (lo < hi) {
      int mid = (lo + hi + 1) / 2;
      if ((int64_t)c->h_row_ptr[mid] - start <= budget) lo = mid;
      else hi = mid - 1;
    }
    int b = std::max(lo, a + 1);
    p.bounds.push_back(b);
    a = b;
  }
  if (n == 0) p.bounds.push_back(0);
  for (size_t q = 0; q + 1 < p.bounds.size(); ++q) {
    p.maxE = std::max<int64_t>(p.maxE, (int64_t)c->h_row_ptr[p.bounds[q + 1]] - c->h_row_ptr[p.bounds[q]]);
    p.maxA = std::max<int64_t>(p.maxA, p.bounds[q + 1] - p.bounds[q]);
  }
  return p;
}

// The device work of one evaluation (no host synchronisation, no allocation:
// it can be captured into a CUDA graph).
allegro_status run_plan(allegro_ctx* c, const Plan& p, const WS& w, bool backward) {
  const int n = (int)c->n_atoms;
  const int64_t E = c->n_edges;
  CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  allegro_status s;
  for (size_t q = 0; q + 1 < p.bounds.size(); ++q) {
    int a0 = p.bounds[q], a1 = p.bounds[q + 1];
    int e0 = c->h_row_ptr[a0], e1 = c->h_row_ptr[a1];
    if (c->generic)
      s = bf16_storage(c) ? run_chunk_gen<bf16>(c, w, a0, a1, e0, e1, backward)
                                         : run_chunk_gen<float>(c, w, a0, a1, e0, e1, backward);
    else
      s = (c->prec == ALLEGRO_PREC_BF16) ? run_chunk<bf16>(c, w, a0, a1, e0, e1, backward)
                                         : run_chunk<float>(c, w, a0, a1, e0, e1, backward);
    if (s != ALLEGRO_OK) return s;
    CUDA_TRY(c, cudaGetLastError());
  }
  {
    ProfScope ps(c, "atom_reduce", 0.0, (double)E * (backward ? 60.0 : 4.0) + (double)n * (backward ? 128.0 : 16.0));
    atom_reduce(n, (int)std::min<int64_t>(c->n_centres, n), c->d_row_ptr, c->d_col_ptr, c->d_col_edge, c->d_Ee, c->d_g, c->d_ed, c->d_species, c->d_sigma,
                c->d_mu, backward, c->d_Eatom, c->d_F, c->d_Wat, c->d_ei, c->d_ej, c->arch, c->stream);
  }
  {
    ProfScope ps(c, "struct_reduce", 0.0, (double)n * (backward ? 104.0 : 8.0));
    struct_reduce(c->nstruct, c->d_offs, c->d_Eatom, c->d_Wat, c->d_F, backward, c->d_Eout, c->d_Wout, c->d_err,
                  c->d_red_scratch, n, c->stream);
  }
  CUDA_TRY(c, cudaGetLastError());
  return ALLEGRO_OK;
}

// One evaluation with the context's current launch configuration: eager, or
// through the cached CUDA graph when graphs are on and nothing it depends on
// changed (chunking, buffer addresses, sizes, configuration, stream).  A graph
// is captured the second time the same key is seen (the first run is eager,
// so one-time set-up such as kernel attributes never happens under capture).
allegro_status evaluate_once(allegro_ctx* c, bool backward) {
  const int64_t budget = c->chunk_edges_user > 0 ? c->chunk_edges_user : c->tune.chunk_edges;
  Plan p = plan_chunks(c, budget);
  WS w;
  allegro_status s = ensure_ws(c, p.maxE, p.maxA, &w);
  if (s != ALLEGRO_OK) return s;
  if (!c->use_graphs || c->prof.on) return run_plan(c, p, w, backward);
  allegro_ctx::GraphKey key;
  key.bounds = p.bounds;
  for (int b : p.bounds) key.bounds.push_back(c->h_row_ptr[b]);   // edge offsets of the chunks too
  key.bounds.push_back((int)c->n_centres);
  key.ptrs = {c->d_row_ptr, c->d_col_ptr, c->d_col_edge, c->d_ej, c->d_ei, c->d_eS, c->d_ed, c->d_Ee, c->d_g,
              c->d_species, c->d_Eatom, c->d_F, c->d_Wat, c->d_offs, c->d_Eout, c->d_Wout, c->d_err,
              c->d_red_scratch, c->ws, c->arch.pair_basis, c->arch.zbl, c->d_atom_struct};
  key.n_atoms = c->n_atoms; key.n_edges = c->n_edges; key.nstruct = c->nstruct; key.backward = backward;
  key.chunk = budget; key.chain_mask = c->tune.chain_mask; key.epq = c->tune.epq_wide; key.stream = c->stream;
  if (c->graph_exec && key == c->graph_key) {
    CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += c->graph_launches;
    ++c->graph_replays;
    return ALLEGRO_OK;
  }
  if (!(key == c->seen_key)) {   // first sight of this key: eager
    c->seen_key = key;
    return run_plan(c, p, w, backward);
  }
  const int64_t l0 = c->launches;
  CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  s = run_plan(c, p, w, backward);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (s != ALLEGRO_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return s;
  }
  if (e != cudaSuccess || !graph) {
    cudaGetLastError();
    return fail(c, ALLEGRO_E_CUDA, "stream capture of the evaluation failed: %s", cudaGetErrorString(e));
  }
  bool updated = false;
  if (c->graph_exec) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(c->graph_exec, graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
  }
  if (!updated) {
    e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      c->graph_exec = nullptr;
      return fail(c, ALLEGRO_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
  }
  cudaGraphDestroy(graph);
  c->graph_key = key;
  c->graph_launches = c->launches - l0;
  CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, c->stream));
  return ALLEGRO_OK;
}

// Shape bucket of the autotuner: precision-independent sizes at quarter-octave
// resolution, pass kind, single or batched.
std::string tune_bucket(const allegro_ctx* c, bool backward) {
  char b[96];
  const int qe = (int)std::lround(4.0 * std::log2((double)std::max<int64_t>(c->n_edges, 1)));
  const int qa = (int)std::lround(4.0 * std::log2((double)std::max<int64_t>(c->n_atoms, 1)));
  snprintf(b, sizeof b, "E2^%.2f/N2^%.2f/%s/%s", qe / 4.0, qa / 4.0, backward ? "EF" : "E",
           c->nstruct > 1 ? "batched" : "single");
  return b;
}

std::string tune_name(const allegro_ctx::Tune& t) {
  char b[96];
  snprintf(b, sizeof b, "chunk=%lld,chain=0x%02x,epq=%d", (long long)t.chunk_edges, t.chain_mask, t.epq_wide);
  return b;
}

// Autotuner: the first evaluation of each shape bucket times candidate launch
// configurations by coordinate descent (edges per chunk; each fused layer pair
// on or off; epilogue warps of the arithmetic single GEMMs), each candidate
// once after one untimed warm-up of the defaults, with CUDA events on the
// context's stream, and keeps the fastest for the bucket.  Every candidate
// computes the same function (chunking and pair fusion change only where
// intermediates live), so the outputs of the final evaluation are the model's.
allegro_status autotune(allegro_ctx* c, bool backward, allegro_ctx::TuneRec* rec) {
  allegro_ctx::Tune best;     // defaults
  cudaEvent_t ev[2];
  CUDA_TRY(c, cudaEventCreate(&ev[0]));
  CUDA_TRY(c, cudaEventCreate(&ev[1]));
  auto time_cfg = [&](const allegro_ctx::Tune& t, double* ms) -> allegro_status {
    c->tune = t;
    cudaEventRecord(ev[0], c->stream);
    allegro_status s = evaluate_once(c, backward);
    cudaEventRecord(ev[1], c->stream);
    if (s != ALLEGRO_OK) return s;
    CUDA_TRY(c, cudaEventSynchronize(ev[1]));
    float f = 0.0f;
    CUDA_TRY(c, cudaEventElapsedTime(&f, ev[0], ev[1]));
    *ms = f;
    rec->trials.push_back({tune_name(t), (double)f});
    return ALLEGRO_OK;
  };
  const bool saved_graphs = c->use_graphs;
  c->use_graphs = false;
  allegro_status s;
  double best_ms = 0.0, ms = 0.0;
  c->tune = best;
  if ((s = evaluate_once(c, backward)) != ALLEGRO_OK) goto done;   // warm-up
  if ((s = time_cfg(best, &best_ms)) != ALLEGRO_OK) goto done;
  {
    // edges per chunk: the largest that fits, then 1/2, 1/4 and 1/8 of the list
    const int64_t E = std::max<int64_t>(c->n_edges, 1);
    for (int64_t div : {2, 4, 8}) {
      allegro_ctx::Tune t = best;
      t.chunk_edges = std::max<int64_t>(E / div, 1 << 16);
      if (t.chunk_edges >= E) continue;
      if ((s = time_cfg(t, &ms)) != ALLEGRO_OK) goto done;
      if (ms < best_ms) { best = t; best_ms = ms; }
    }
    if (c->prec == ALLEGRO_PREC_BF16) {
      for (int k = 0; k < 6; ++k) {   // each fused layer pair on or off
        allegro_ctx::Tune t = best;
        t.chain_mask ^= 1 << k;
        if ((s = time_cfg(t, &ms)) != ALLEGRO_OK) goto done;
        if (ms < best_ms) { best = t; best_ms = ms; }
      }
      allegro_ctx::Tune t = best;
      t.epq_wide = best.epq_wide == 4 ? 2 : 4;
      if ((s = time_cfg(t, &ms)) != ALLEGRO_OK) goto done;
      if (ms < best_ms) { best = t; best_ms = ms; }
    }
  }
done:
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  c->use_graphs = saved_graphs;
  c->tune = best;
  rec->best = best;
  return s;
}

allegro_status evaluate(allegro_ctx* c, bool backward) {
  if (c->autotune) {
    const std::string b = tune_bucket(c, backward);
    auto it = c->tuned.find(b);
    if (it == c->tuned.end()) {
      allegro_ctx::TuneRec rec;
      allegro_status s = autotune(c, backward, &rec);
      if (s != ALLEGRO_OK) return s;
      it = c->tuned.emplace(b, rec).first;
    }
    c->tune = it->second.best;
  }
  return evaluate_once(c, backward);
}

allegro_status copy_out(allegro_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!dst || bytes == 0) return ALLEGRO_OK;
  cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, k, c->stream));
  return ALLEGRO_OK;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

allegro_status allegro_create(const void* weights_blob, size_t blob_bytes, const int32_t* species_map,
                              int32_t n_types, double r_c, int32_t precision, int32_t device, allegro_ctx** out) {
  if (!out) return ALLEGRO_E_INVALID;
  *out = nullptr;
  if (!weights_blob || blob_bytes == 0) return ALLEGRO_E_INVALID;
  if (precision != ALLEGRO_PREC_FP32 && precision != ALLEGRO_PREC_BF16 && precision != ALLEGRO_PREC_TF32 &&
      precision != ALLEGRO_PREC_FP8)
    return ALLEGRO_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ALLEGRO_E_CUDA;
  }
  allegro_ctx* c = new allegro_ctx();
  c->device = device;
  c->prec = precision;
  auto bail = [&](allegro_status s) {
    fprintf(stderr, "allegro_create: %s\n", c->err.c_str());
    allegro_destroy(c);
    return s;
  };
  if (cudaSetDevice(device) != cudaSuccess) return bail(fail(c, ALLEGRO_E_CUDA, "cudaSetDevice failed"));
  if (precision == ALLEGRO_PREC_BF16 || precision == ALLEGRO_PREC_TF32 || precision == ALLEGRO_PREC_FP8) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    if (prop.major != 10 || prop.minor != 3)
      return bail(fail(c, ALLEGRO_E_INVALID, "BF16 path needs sm_103 (found sm_%d%d)", prop.major, prop.minor));
    std::string why;
    if (!gemm_tc_init(&why)) return bail(fail(c, ALLEGRO_E_CUDA, "%s", why.c_str()));
  }
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(c, ALLEGRO_E_CUDA, "cudaStreamCreate failed"));
  c->stream = c->own_stream;
  allegro_status s = load_model(c, weights_blob, blob_bytes);
  if (s != ALLEGRO_OK) return bail(s);
  if (precision == ALLEGRO_PREC_FP8 && cudaMalloc(&c->d_amax, kAmaxSlots * sizeof(unsigned)) != cudaSuccess)
    return bail(fail(c, ALLEGRO_E_OOM, "amax slots"));
  if (r_c > 0 && fabs(r_c - c->arch.rc) > 1e-12 * c->arch.rc)
    return bail(fail(c, ALLEGRO_E_INVALID, "r_c %g differs from the model cutoff %g", r_c, c->arch.rc));
  // species map
  if (species_map) {
    if (n_types <= 0) return bail(fail(c, ALLEGRO_E_INVALID, "n_types must be positive"));
    for (int t = 0; t < n_types; ++t) {
      if (species_map[t] < 0 || species_map[t] >= c->arch.ns)
        return bail(fail(c, ALLEGRO_E_INVALID, "species_map[%d] = %d out of range", t, species_map[t]));
      c->species_map.push_back(species_map[t]);
    }
  } else {
    for (int t = 0; t < c->arch.ns; ++t) c->species_map.push_back(t);
  }
  c->nmap = (int)c->species_map.size();
  if (cudaMalloc(&c->d_map, c->nmap * 4) != cudaSuccess ||
      cudaMemcpy(c->d_map, c->species_map.data(), c->nmap * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(c, ALLEGRO_E_OOM, "species map upload failed"));
  if (cudaMalloc(&c->d_err, 16) != cudaSuccess || cudaMalloc(&c->d_total, 16) != cudaSuccess ||
      cudaMalloc(&c->d_minmax, 12 * 8) != cudaSuccess || cudaMalloc(&c->d_red_scratch, 12 * 1024 * 8) != cudaSuccess)
    return bail(fail(c, ALLEGRO_E_OOM, "scratch allocation failed"));
  cudaMemset(c->d_err, 0, 16);
  *out = c;
  return ALLEGRO_OK;
}

allegro_status allegro_set_stream(allegro_ctx* c, void* stream) {
  if (!c) return ALLEGRO_E_INVALID;
  c->stream = stream ? reinterpret_cast<cudaStream_t>(stream) : c->own_stream;
  return ALLEGRO_OK;
}

allegro_status allegro_set_pair_cutoffs(allegro_ctx* c, const double* pair_rc, int32_t n_species) {
  if (!c) return ALLEGRO_E_INVALID;
  cudaSetDevice(c->device);
  c->have_nb = false;
  if (!pair_rc) {
    c->arch.pair_basis = nullptr;
    c->arch.pair_rc2 = nullptr;
    return ALLEGRO_OK;
  }
  const int ns = c->arch.ns;
  if (n_species != ns) return fail(c, ALLEGRO_E_INVALID, "n_species %d differs from the model's %d", n_species, ns);
  std::vector<float> basis(2 * (size_t)ns * ns);
  std::vector<double> rc2((size_t)ns * ns);
  for (int q = 0; q < ns * ns; ++q) {
    const double rc = pair_rc[q];
    // the cell grid and the prefilter band are built for the model cutoff, the largest allowed
    if (!(rc > 0.0) || !(rc <= c->arch.rc))
      return fail(c, ALLEGRO_E_INVALID, "pair cutoff [%d][%d] = %g outside (0, %g]", q / ns, q % ns, rc, c->arch.rc);
    basis[2 * q] = (float)(1.0 / rc);
    basis[2 * q + 1] = (float)std::sqrt(2.0 / rc);
    rc2[q] = rc * rc;
  }
  if (!c->d_pair_basis) {
    CUDA_TRY(c, cudaMalloc(&c->d_pair_basis, 2 * sizeof(float) * kMaxSpecies * kMaxSpecies));
    CUDA_TRY(c, cudaMalloc(&c->d_pair_rc2, sizeof(double) * kMaxSpecies * kMaxSpecies));
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_pair_basis, basis.data(), basis.size() * sizeof(float), cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_pair_rc2, rc2.data(), rc2.size() * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->arch.pair_basis = c->d_pair_basis;
  c->arch.pair_rc2 = c->d_pair_rc2;
  return ALLEGRO_OK;
}

allegro_status allegro_set_zbl(allegro_ctx* c, const int32_t* atomic_numbers, int32_t n_species) {
  if (!c) return ALLEGRO_E_INVALID;
  cudaSetDevice(c->device);
  if (!atomic_numbers) {
    c->arch.zbl = nullptr;
    return ALLEGRO_OK;
  }
  const int ns = c->arch.ns;
  if (n_species != ns) return fail(c, ALLEGRO_E_INVALID, "n_species %d differs from the model's %d", n_species, ns);
  for (int q = 0; q < ns; ++q)
    if (atomic_numbers[q] < 1 || atomic_numbers[q] > 118)
      return fail(c, ALLEGRO_E_INVALID, "atomic number of species %d = %d outside 1..118", q, atomic_numbers[q]);
  // Coulomb constant e^2 / (4 pi eps_0) in eV A, Bohr radius in A, universal screening length
  const double ke = 14.399645, a0 = 0.529177;
  std::vector<float> t(2 * (size_t)ns * ns);
  for (int za = 0; za < ns; ++za)
    for (int zb = 0; zb < ns; ++zb) {
      const double Za = atomic_numbers[za], Zb = atomic_numbers[zb];
      const double as = 0.8854 * a0 / (std::pow(Za, 0.23) + std::pow(Zb, 0.23));
      t[2 * ((size_t)za * ns + zb)] = (float)(0.5 * ke * Za * Zb);
      t[2 * ((size_t)za * ns + zb) + 1] = (float)(1.0 / as);
    }
  if (!c->d_zbl) CUDA_TRY(c, cudaMalloc(&c->d_zbl, 2 * sizeof(float) * kMaxSpecies * kMaxSpecies));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_zbl, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->arch.zbl = c->d_zbl;
  return ALLEGRO_OK;
}

allegro_status allegro_reserve(allegro_ctx* c, int64_t atom_cap, int64_t edge_cap, int32_t fixed,
                               int64_t chunk_edges) {
  if (!c || atom_cap < 0 || edge_cap < 0 || chunk_edges < 0) return ALLEGRO_E_INVALID;
  cudaSetDevice(c->device);
  c->fixed = fixed != 0;
  c->atom_cap = atom_cap;
  c->edge_cap = edge_cap;
  c->chunk_edges_user = chunk_edges;
  if (atom_cap > 0) {
    allegro_status s = stage_atoms(c, 0, nullptr, nullptr);
    if (s != ALLEGRO_OK) return s;
    Caps& k = caps_of(c);
    CUDA_TRY(c, grow(c->d_pos, k.pos, 3 * atom_cap));
  }
  if (edge_cap > 0) {
    bool f = c->fixed;
    c->fixed = false;
    allegro_status s = ensure_edges(c, edge_cap);
    c->fixed = f;
    if (s != ALLEGRO_OK) return s;
  }
  return ALLEGRO_OK;
}

// The cell-list search of one structure at `radius` (the model cutoff, or the
// cutoff plus a Verlet skin for a candidate list), the per-pair table applied
// only when `use_pair` is set.
static allegro_status build_single(allegro_ctx* c, int64_t n_atoms, const double* pos, const int32_t* types,
                                   const double* cell, const uint8_t* pbc, int64_t* n_edges_out, double radius,
                                   bool use_pair, int64_t n_centres = -1) {
  if (!c) return ALLEGRO_E_INVALID;
  c->have_nb = false;
  if (n_atoms < 0 || n_atoms > 1000000000LL) return fail(c, ALLEGRO_E_INVALID, "bad n_atoms");
  if (n_atoms > 0 && (!pos || !types)) return fail(c, ALLEGRO_E_INVALID, "pos and types are required");
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  const int n = (int)n_atoms;
  allegro_status s = stage_atoms(c, n, pos, types);
  if (s != ALLEGRO_OK) return s;
  if ((s = ensure_structs(c, 1)) != ALLEGRO_OK) return s;
  int64_t hoffs[2] = {0, n};
  CUDA_TRY(c, cudaMemcpyAsync(c->d_offs, hoffs, sizeof hoffs, cudaMemcpyHostToDevice, st));
  c->nstruct = 1;
  c->batched = false;

  // cell and periodicity (host copies)
  double hcell[9] = {0};
  uint8_t hpbc[3] = {0, 0, 0};
  if (cell) {
    if (is_device_ptr(cell)) CUDA_TRY(c, cudaMemcpy(hcell, cell, sizeof hcell, cudaMemcpyDeviceToHost));
    else memcpy(hcell, cell, sizeof hcell);
    for (double v : hcell)
      if (!std::isfinite(v)) return fail(c, ALLEGRO_E_INVALID, "cell is not finite");
  }
  if (pbc) {
    if (is_device_ptr(pbc)) CUDA_TRY(c, cudaMemcpy(hpbc, pbc, 3, cudaMemcpyDeviceToHost));
    else memcpy(hpbc, pbc, 3);
  } else if (cell) {
    hpbc[0] = hpbc[1] = hpbc[2] = 1;
  }
  CellGrid g{};
  g.n_centres = (n_centres < 0 || n_centres > n) ? n : (int)n_centres;
  const double rc = radius, rcm = rc * (1.0 + 1e-6);
  const double* pair_rc2 = use_pair ? c->arch.pair_rc2 : nullptr;
  memcpy(c->h_cell, hcell, sizeof hcell);
  double width[3] = {1, 1, 1};
  if (cell) {
    if (!invert3(hcell, g.inv)) return fail(c, ALLEGRO_E_INVALID, "cell is singular");
    widths_of(hcell, width);
    memcpy(g.cell, hcell, sizeof hcell);
  } else {
    for (int k = 0; k < 3; ++k) {
      if (hpbc[k]) return fail(c, ALLEGRO_E_INVALID, "a periodic axis needs a cell");
      g.inv[k * 3 + k] = 1.0;
    }
  }
  bool any_np = false;
  for (int k = 0; k < 3; ++k) {
    g.pbc[k] = hpbc[k] ? 1 : 0;
    any_np |= !g.pbc[k];
  }
  double hmm[6] = {0, 0, 0, 0, 0, 0};
  if (any_np && n > 0) {
    nb_minmax_frac(c->d_pos, n, g.inv, c->d_minmax, st);
    CUDA_TRY(c, cudaMemcpyAsync(hmm, c->d_minmax, 6 * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
  }
  int64_t ncell = 1;
  for (int k = 0; k < 3; ++k) {
    double ext;
    if (g.pbc[k]) {
      ext = width[k];
      g.lo[k] = 0; g.span[k] = 1;
    } else {
      double lo = hmm[k], hi = hmm[3 + k];
      if (!(hi >= lo)) { lo = 0; hi = 0; }
      g.lo[k] = lo;
      g.span[k] = (hi - lo) * (1.0 + 1e-9) + 1e-300;
      ext = (hi - lo) * (cell ? width[k] : 1.0);
    }
    int64_t nk = (int64_t)floor(ext / rcm);
    nk = std::max<int64_t>(1, std::min<int64_t>(nk, 4096));
    g.n[k] = (int)nk;
    g.R[k] = (g.pbc[k] && ext / nk < rcm) ? (int)ceil(rcm * nk / ext) : 1;
    ncell *= nk;
  }
  // very sparse grids: coarsen (larger cells stay >= r_c wide, so the stencil still covers r_c)
  const int64_t max_cells = std::max<int64_t>(4 * (int64_t)n, 64);
  while (ncell > max_cells) {
    int kmax = 0;
    for (int k = 1; k < 3; ++k) if (g.n[k] > g.n[kmax]) kmax = k;
    g.n[kmax] = std::max(1, g.n[kmax] / 2);
    ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
  }
  Caps& k = caps_of(c);
  CUDA_TRY(c, grow(c->d_cell_count, k.cc, ncell + 1));
  CUDA_TRY(c, grow(c->d_cell_start, k.cs, ncell + 1));
  CUDA_TRY(c, grow(c->d_cell_cursor, k.ccur, ncell + 1));
  size_t need_tmp = scan_tmp_bytes((int)std::max<int64_t>(ncell, n)) + 4096;
  if (need_tmp > c->scan_tmp_cap) {
    if (c->d_scan_tmp) cudaFree(c->d_scan_tmp);
    c->d_scan_tmp = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_scan_tmp, need_tmp * 2));
    c->scan_tmp_cap = need_tmp * 2;
  }
  CUDA_TRY(c, cudaMemsetAsync(c->d_cell_count, 0, (size_t)(ncell + 1) * 4, st));
  {
    ProfScope ps(c, "nb_bin_sort", 0.0, (double)n * 80 + (double)ncell * 16, 7);
    nb_bin(c->d_pos, n, g, c->d_cell_of, c->d_wrap, c->d_cell_count, st);
    exclusive_scan_i32(c->d_cell_count, c->d_cell_start, (int)ncell, nullptr, c->d_scan_tmp, c->scan_tmp_cap, st);
    CUDA_TRY(c, cudaMemsetAsync(c->d_cell_cursor, 0, (size_t)(ncell + 1) * 4, st));
    nb_place(c->d_cell_of, n, c->d_cell_start, c->d_cell_cursor, c->d_sorted, st);
    nb_sort_cells(c->d_cell_start, (int)ncell, c->d_sorted, st);
    nb_pos4(c->d_pos, c->d_species, n, g, c->d_wrap, c->d_sorted, c->d_pos4, c->d_pw, c->d_wraps, st);
  }
  // Error band of the float32 prefilter: bound X on |wrapped coordinate| and
  // |image offset|, per-component error <= 8 ulp(X), squared-distance error
  // <= 2 sqrt3 r_c delta + 3 delta^2 + rounding of the sum; safety factor 4.
  float band;
  {
    double X = 0.0, Xoff = 0.0;
    for (int k3 = 0; k3 < 3; ++k3) {
      double Fk = g.pbc[k3] ? 1.0 : std::max(fabs(hmm[k3]), fabs(hmm[3 + k3])) + 1.0;
      double rowlen = cell ? sqrt(hcell[3 * k3] * hcell[3 * k3] + hcell[3 * k3 + 1] * hcell[3 * k3 + 1] +
                                  hcell[3 * k3 + 2] * hcell[3 * k3 + 2])
                           : 1.0;
      X += Fk * rowlen;
      Xoff += (g.pbc[k3] ? g.R[k3] : 0) * rowlen;
    }
    const double delta = 8.0 * (X + Xoff) * std::ldexp(1.0, -23);
    const double bd = 4.0 * (2.0 * sqrt(3.0) * rc * delta + 3.0 * delta * delta + 1e-6 * rc * rc);
    band = (float)bd;
    if (!(band > 0) || !std::isfinite(band) || band > 0.25 * rc * rc) band = 1e30f;   // prefilter off
  }
  const double rc2 = rc * rc;
  {
    ProfScope ps(c, "nb_search_count", 0.0, (double)n * 64, 4);
    nb_search(false, c->d_pos, n, g, c->d_cell_of, c->d_wraps, c->d_cell_start, c->d_sorted, c->d_pos4, c->d_pw, rc2,
              band, pair_rc2, c->arch.ns, c->d_count,
              nullptr, nullptr, nullptr, nullptr, nullptr, c->d_err, st);
    exclusive_scan_i32(c->d_count, c->d_row_ptr, n, nullptr, c->d_scan_tmp, c->scan_tmp_cap, st);
  }
  int hE = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&hE, c->d_row_ptr + n, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  CUDA_TRY(c, cudaGetLastError());
  if (hE < 0) return fail(c, ALLEGRO_E_CAPACITY, "edge count overflows int32");
  if ((s = ensure_edges(c, hE)) != ALLEGRO_OK) return s;
  {
    ProfScope ps(c, "nb_search_fill", 0.0, (double)hE * 44 + (double)n * 64);
    nb_search(true, c->d_pos, n, g, c->d_cell_of, c->d_wraps, c->d_cell_start, c->d_sorted, c->d_pos4, c->d_pw, rc2,
              band, pair_rc2, c->arch.ns, nullptr,
              c->d_row_ptr, c->d_ej, c->d_ei, c->d_eS, c->d_ed, c->d_err, st);
  }
  if ((s = finish_neighbors(c, n, hE)) != ALLEGRO_OK) return s;
  c->n_centres = g.n_centres;
  if (n_edges_out) *n_edges_out = hE;
  return ALLEGRO_OK;
}

allegro_status allegro_neighbors(allegro_ctx* c, int64_t n_atoms, const double* pos, const int32_t* types,
                                 const double* cell, const uint8_t* pbc, int64_t* n_edges_out) {
  if (!c) return ALLEGRO_E_INVALID;
  return build_single(c, n_atoms, pos, types, cell, pbc, n_edges_out, c->arch.rc, true);
}

allegro_status allegro_neighbors_local(allegro_ctx* c, int64_t n_local, int64_t n_atoms, const double* pos,
                                       const int32_t* types, const double* cell, const uint8_t* pbc,
                                       int64_t* n_edges_out) {
  if (!c) return ALLEGRO_E_INVALID;
  if (n_local < 0 || n_local > n_atoms) return fail(c, ALLEGRO_E_INVALID, "n_local must be in [0, n_atoms]");
  return build_single(c, n_atoms, pos, types, cell, pbc, n_edges_out, c->arch.rc, true, n_local);
}

allegro_status allegro_neighbors_batched(allegro_ctx* c, int32_t n_struct, const int64_t* atom_offsets,
                                         const double* pos, const int32_t* types, const double* cells,
                                         const uint8_t* pbc, int64_t* n_edges_out) {
  if (!c) return ALLEGRO_E_INVALID;
  c->have_nb = false;
  if (n_struct < 1 || !atom_offsets) return fail(c, ALLEGRO_E_INVALID, "n_struct >= 1 and atom_offsets required");
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  std::vector<int64_t> offs((size_t)n_struct + 1);
  if (is_device_ptr(atom_offsets))
    CUDA_TRY(c, cudaMemcpy(offs.data(), atom_offsets, offs.size() * 8, cudaMemcpyDeviceToHost));
  else memcpy(offs.data(), atom_offsets, offs.size() * 8);
  if (offs[0] != 0) return fail(c, ALLEGRO_E_INVALID, "atom_offsets[0] must be 0");
  for (int b = 0; b < n_struct; ++b)
    if (offs[b + 1] < offs[b]) return fail(c, ALLEGRO_E_INVALID, "atom_offsets must be non-decreasing");
  const int64_t n64 = offs[n_struct];
  if (n64 > 1000000000LL) return fail(c, ALLEGRO_E_INVALID, "too many atoms");
  const int n = (int)n64;
  if (n > 0 && (!pos || !types)) return fail(c, ALLEGRO_E_INVALID, "pos and types are required");
  allegro_status s = stage_atoms(c, n, pos, types);
  if (s != ALLEGRO_OK) return s;
  if ((s = ensure_structs(c, n_struct)) != ALLEGRO_OK) return s;
  std::vector<double> hc;
  std::vector<int> hp((size_t)3 * n_struct, 0), hn((size_t)3 * n_struct, 0);
  if (cells) {
    hc.resize((size_t)9 * n_struct);
    if (is_device_ptr(cells)) CUDA_TRY(c, cudaMemcpy(hc.data(), cells, hc.size() * 8, cudaMemcpyDeviceToHost));
    else memcpy(hc.data(), cells, hc.size() * 8);
  }
  std::vector<uint8_t> hpb((size_t)3 * n_struct, cells ? 1 : 0);
  if (pbc) {
    if (is_device_ptr(pbc)) CUDA_TRY(c, cudaMemcpy(hpb.data(), pbc, hpb.size(), cudaMemcpyDeviceToHost));
    else memcpy(hpb.data(), pbc, hpb.size());
  }
  const double rc = c->arch.rc;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_offs, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, st));
  // image ranges: |S_k| <= ceil(r_c / w_k + span_k), span_k the spread of the
  // structure's fractional coordinates (positions need not be wrapped)
  std::vector<double> hinv((size_t)9 * n_struct, 0.0), hspan((size_t)3 * n_struct, 0.0);
  if (cells) {
    for (int b = 0; b < n_struct; ++b)
      if (!invert3(&hc[9 * (size_t)b], &hinv[9 * (size_t)b])) return fail(c, ALLEGRO_E_INVALID, "cell %d is singular", b);
    double* d_inv = nullptr;
    double* d_span = nullptr;
    CUDA_TRY(c, cudaMalloc(&d_inv, hinv.size() * 8));
    CUDA_TRY(c, cudaMalloc(&d_span, hspan.size() * 8));
    cudaMemcpyAsync(d_inv, hinv.data(), hinv.size() * 8, cudaMemcpyHostToDevice, st);
    nb_struct_span(c->d_pos, c->d_offs, d_inv, n_struct, d_span, st);
    cudaMemcpyAsync(hspan.data(), d_span, hspan.size() * 8, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(d_inv);
    cudaFree(d_span);
    if (e != cudaSuccess) return fail(c, ALLEGRO_E_CUDA, "span: %s", cudaGetErrorString(e));
  }
  for (int b = 0; b < n_struct; ++b) {
    double w[3] = {1, 1, 1};
    if (cells) widths_of(&hc[9 * (size_t)b], w);
    for (int k = 0; k < 3; ++k) {
      hp[3 * b + k] = hpb[3 * b + k] ? 1 : 0;
      if (hp[3 * b + k] && !cells) return fail(c, ALLEGRO_E_INVALID, "a periodic axis needs a cell");
      hn[3 * b + k] = hp[3 * b + k] ? (int)ceil(rc / w[k] + hspan[3 * b + k]) : 0;
    }
  }
  if (cells) CUDA_TRY(c, cudaMemcpyAsync(c->d_cells, hc.data(), hc.size() * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_pbc, hp.data(), hp.size() * 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_nimg, hn.data(), hn.size() * 4, cudaMemcpyHostToDevice, st));
  atom_struct_kernel<<<n_struct, 128, 0, st>>>(c->d_offs, n_struct, c->d_atom_struct);
  const double rc2 = rc * rc;
  nb_bruteforce_batched(false, c->d_pos, c->d_offs, n_struct, cells ? c->d_cells : nullptr, c->d_pbc, c->d_nimg, rc2,
                        c->d_species, c->arch.pair_rc2, c->arch.ns, c->d_atom_struct, n, c->d_count, nullptr, nullptr, nullptr, nullptr, nullptr, c->d_err, st);
  exclusive_scan_i32(c->d_count, c->d_row_ptr, n, nullptr, c->d_scan_tmp, c->scan_tmp_cap, st);
  int hE = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&hE, c->d_row_ptr + n, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  CUDA_TRY(c, cudaGetLastError());
  if ((s = ensure_edges(c, hE)) != ALLEGRO_OK) return s;
  nb_bruteforce_batched(true, c->d_pos, c->d_offs, n_struct, cells ? c->d_cells : nullptr, c->d_pbc, c->d_nimg, rc2,
                        c->d_species, c->arch.pair_rc2, c->arch.ns, c->d_atom_struct, n, nullptr, c->d_row_ptr, c->d_ej, c->d_ei, c->d_eS, c->d_ed, c->d_err, st);
  if ((s = finish_neighbors(c, n, hE)) != ALLEGRO_OK) return s;
  c->nstruct = n_struct;
  c->batched = true;
  if (n_edges_out) *n_edges_out = hE;
  return ALLEGRO_OK;
}

allegro_status allegro_energy_forces(allegro_ctx* c, double* E_total, double* E_atom, double* F, double* virial) {
  if (!c) return ALLEGRO_E_INVALID;
  if (!E_total) return fail(c, ALLEGRO_E_INVALID, "E_total is required");
  if (!c->have_nb) return fail(c, ALLEGRO_E_STATE, "allegro_neighbors must succeed before energy_forces");
  cudaSetDevice(c->device);
  const bool backward = (F != nullptr) || (virial != nullptr);
  allegro_status s = evaluate(c, backward);
  if (s != ALLEGRO_OK) return s;
  const size_t n = (size_t)c->n_atoms, B = (size_t)c->nstruct;
  if ((s = copy_out(c, E_total, c->d_Eout, B * 8)) != ALLEGRO_OK) return s;
  if ((s = copy_out(c, E_atom, c->d_Eatom, n * 8)) != ALLEGRO_OK) return s;
  if (F && (s = copy_out(c, F, c->d_F, n * 3 * 8)) != ALLEGRO_OK) return s;
  if (virial && (s = copy_out(c, virial, c->d_Wout, B * 9 * 8)) != ALLEGRO_OK) return s;
  int err = 0;
  if ((s = read_err(c, &err)) != ALLEGRO_OK) return s;
  if (err & kErrTimeout) return fail(c, ALLEGRO_E_TIMEOUT, "a bounded device wait expired; results are invalid");
  if (err & kErrNonFinite) return fail(c, ALLEGRO_E_NONFINITE, "non-finite energy or force");
  return ALLEGRO_OK;
}

allegro_status allegro_md_verlet(allegro_ctx* c, int64_t n_atoms, double* pos, double* vel, const int32_t* types,
                                 const double* masses, int32_t n_types, const double* cell, const uint8_t* pbc,
                                 double dt, int64_t n_steps, double* E_pot, double* E_kin) {
  if (!c) return ALLEGRO_E_INVALID;
  if (n_atoms < 1 || n_atoms > 1000000000LL || !pos || !vel || !types || !masses || n_types < 1 || n_steps < 0 ||
      !(dt > 0) || !std::isfinite(dt))
    return fail(c, ALLEGRO_E_INVALID, "md_verlet: bad arguments");
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  const int n = (int)n_atoms;
  if (n_atoms > c->md_atoms) {
    cudaFree(c->d_md_pos); cudaFree(c->d_md_vel); cudaFree(c->d_md_invm); cudaFree(c->d_md_types);
    cudaFree(c->d_sk_ref);
    c->d_md_pos = c->d_md_vel = c->d_md_invm = c->d_sk_ref = nullptr;
    c->d_md_types = nullptr;
    c->md_atoms = 0;
    CUDA_TRY(c, cudaMalloc(&c->d_md_pos, (size_t)n * 24));
    CUDA_TRY(c, cudaMalloc(&c->d_md_vel, (size_t)n * 24));
    CUDA_TRY(c, cudaMalloc(&c->d_md_invm, (size_t)n * 8));
    CUDA_TRY(c, cudaMalloc(&c->d_md_types, (size_t)n * 4));
    c->md_atoms = n_atoms;
  }
  if (n_steps + 1 > c->md_steps || !c->d_md_part) {
    cudaFree(c->d_md_E); cudaFree(c->d_md_K); cudaFree(c->d_md_part); cudaFree(c->d_md_masses);
    c->d_md_E = c->d_md_K = c->d_md_part = c->d_md_masses = nullptr;
    c->md_steps = 0;
    CUDA_TRY(c, cudaMalloc(&c->d_md_E, (size_t)(n_steps + 1) * 8));
    CUDA_TRY(c, cudaMalloc(&c->d_md_K, (size_t)(n_steps + 1) * 8));
    CUDA_TRY(c, cudaMalloc(&c->d_md_part, 256 * 8));
    CUDA_TRY(c, cudaMalloc(&c->d_md_masses, 4096 * 8));
    c->md_steps = n_steps + 1;
  }
  if (n_types > 4096) return fail(c, ALLEGRO_E_INVALID, "md_verlet: too many types");
  auto kind = [](const void* p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
  CUDA_TRY(c, cudaMemcpyAsync(c->d_md_pos, pos, (size_t)n * 24, kind(pos), st));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_md_vel, vel, (size_t)n * 24, kind(vel), st));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_md_types, types, (size_t)n * 4, kind(types), st));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_md_masses, masses, (size_t)n_types * 8, kind(masses), st));
  CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  md_inv_mass(n, c->d_md_types, c->d_md_masses, n_types, c->d_md_invm, c->d_err, st);
  int err = 0;
  allegro_status s = read_err(c, &err);
  if (s != ALLEGRO_OK) return s;
  if (err) return fail(c, ALLEGRO_E_INVALID, "md_verlet: a type has no positive mass");
  // The neighbour list of the current positions: rebuilt by the cell-list
  // search every step, or, with a Verlet skin, filtered from a candidate list
  // built at r_c + skin, rebuilt only once some atom has moved skin/2 since
  // that build (so every pair now within r_c was a candidate; the filter
  // applies the exact rule, so the list equals a rebuild's as a set).
  c->md_rebuilds = 0;
  auto neighbours = [&](bool first) -> allegro_status {
    if (!(c->md_skin > 0.0)) {
      ++c->md_rebuilds;
      return allegro_neighbors(c, n_atoms, c->d_md_pos, c->d_md_types, cell, pbc, nullptr);
    }
    bool rebuild = first;
    if (!rebuild) {
      nb_max_disp2(c->d_md_pos, c->d_sk_ref, n, c->d_maxd, st);
      unsigned long long h = 0;
      CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_maxd, sizeof h, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(c, cudaStreamSynchronize(st));
      double m2 = 0.0;
      memcpy(&m2, &h, sizeof m2);
      rebuild = !(2.0 * sqrt(m2) < c->md_skin * (1.0 - 1e-9));
    }
    allegro_status r;
    if (rebuild) {
      int64_t Ec = 0;
      if ((r = build_single(c, n_atoms, c->d_md_pos, c->d_md_types, cell, pbc, &Ec, c->arch.rc + c->md_skin,
                            false)) != ALLEGRO_OK)
        return r;
      CUDA_TRY(c, regrow(c->d_sk_row, c->sk_row_cap, (int64_t)n + 1));
      CUDA_TRY(c, regrow(c->d_sk_j, c->sk_cap, std::max<int64_t>(Ec, 1)));
      CUDA_TRY(c, regrow(c->d_sk_S, c->sk_S_cap, 3 * std::max<int64_t>(Ec, 1)));
      if (!c->d_sk_ref) CUDA_TRY(c, cudaMalloc(&c->d_sk_ref, (size_t)c->md_atoms * 24));
      if (!c->d_cell9) CUDA_TRY(c, cudaMalloc(&c->d_cell9, 9 * sizeof(double)));
      if (!c->d_maxd) CUDA_TRY(c, cudaMalloc(&c->d_maxd, sizeof(unsigned long long)));
      CUDA_TRY(c, cudaMemcpyAsync(c->d_sk_row, c->d_row_ptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(c, cudaMemcpyAsync(c->d_sk_j, c->d_ej, (size_t)Ec * 4, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(c, cudaMemcpyAsync(c->d_sk_S, c->d_eS, (size_t)Ec * 12, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(c, cudaMemcpyAsync(c->d_sk_ref, c->d_md_pos, (size_t)n * 24, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(c, cudaMemcpyAsync(c->d_cell9, c->h_cell, sizeof c->h_cell, cudaMemcpyHostToDevice, st));
      ++c->md_rebuilds;
    } else if ((r = stage_atoms(c, n, c->d_md_pos, c->d_md_types)) != ALLEGRO_OK) {
      return r;
    }
    c->have_nb = false;
    {
      ProfScope ps(c, "nb_skin_filter", 0.0, (double)n * 64, 2);
      nb_skin_filter(false, c->d_pos, n, c->d_cell9, c->d_sk_row, c->d_sk_j, c->d_sk_S, c->arch.rc * c->arch.rc,
                     c->arch.pair_rc2, c->d_species, c->arch.ns, c->d_count, nullptr, nullptr, nullptr, nullptr,
                     nullptr, st);
      exclusive_scan_i32(c->d_count, c->d_row_ptr, n, nullptr, c->d_scan_tmp, c->scan_tmp_cap, st);
    }
    int hE = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&hE, c->d_row_ptr + n, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    if ((r = ensure_edges(c, hE)) != ALLEGRO_OK) return r;
    {
      ProfScope ps(c, "nb_skin_filter", 0.0, (double)hE * 44 + (double)n * 64);
      nb_skin_filter(true, c->d_pos, n, c->d_cell9, c->d_sk_row, c->d_sk_j, c->d_sk_S, c->arch.rc * c->arch.rc,
                     c->arch.pair_rc2, c->d_species, c->arch.ns, nullptr, c->d_row_ptr, c->d_ej, c->d_ei, c->d_eS,
                     c->d_ed, st);
    }
    CUDA_TRY(c, cudaGetLastError());
    return finish_neighbors(c, n, hE);
  };
  // forces at the initial positions
  if ((s = neighbours(true)) != ALLEGRO_OK) return s;
  if ((s = evaluate(c, true)) != ALLEGRO_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_md_E, c->d_Eout, 8, cudaMemcpyDeviceToDevice, st));
  md_kinetic(n, c->d_md_vel, c->d_md_invm, c->d_md_part, c->d_md_K, st);
  for (int64_t k = 1; k <= n_steps; ++k) {
    md_kick(n, c->d_md_pos, c->d_md_vel, c->d_F, c->d_md_invm, dt, true, st);
    if ((s = neighbours(false)) != ALLEGRO_OK) return s;
    if ((s = evaluate(c, true)) != ALLEGRO_OK) return s;
    md_kick(n, c->d_md_pos, c->d_md_vel, c->d_F, c->d_md_invm, dt, false, st);
    CUDA_TRY(c, cudaMemcpyAsync(c->d_md_E + k, c->d_Eout, 8, cudaMemcpyDeviceToDevice, st));
    md_kinetic(n, c->d_md_vel, c->d_md_invm, c->d_md_part, c->d_md_K + k, st);
  }
  CUDA_TRY(c, cudaGetLastError());
  if ((s = copy_out(c, pos, c->d_md_pos, (size_t)n * 24)) != ALLEGRO_OK) return s;
  if ((s = copy_out(c, vel, c->d_md_vel, (size_t)n * 24)) != ALLEGRO_OK) return s;
  if ((s = copy_out(c, E_pot, c->d_md_E, (size_t)(n_steps + 1) * 8)) != ALLEGRO_OK) return s;
  if ((s = copy_out(c, E_kin, c->d_md_K, (size_t)(n_steps + 1) * 8)) != ALLEGRO_OK) return s;
  if ((s = read_err(c, &err)) != ALLEGRO_OK) return s;
  if (err & kErrTimeout) return fail(c, ALLEGRO_E_TIMEOUT, "a bounded device wait expired; results are invalid");
  if (err & kErrNonFinite) return fail(c, ALLEGRO_E_NONFINITE, "non-finite energy or force");
  return ALLEGRO_OK;
}

allegro_status allegro_set_autotune(allegro_ctx* c, int32_t enable) {
  if (!c) return ALLEGRO_E_INVALID;
  c->autotune = enable != 0;
  if (!c->autotune) c->tune = allegro_ctx::Tune();
  return ALLEGRO_OK;
}

allegro_status allegro_set_graphs(allegro_ctx* c, int32_t enable) {
  if (!c) return ALLEGRO_E_INVALID;
  cudaSetDevice(c->device);
  c->use_graphs = enable != 0;
  if (!c->use_graphs && c->graph_exec) {
    cudaStreamSynchronize(c->stream);
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    c->graph_key = allegro_ctx::GraphKey();
  }
  c->seen_key = allegro_ctx::GraphKey();
  return ALLEGRO_OK;
}

allegro_status allegro_autotune_report(allegro_ctx* c, char* buf, size_t cap) {
  if (!c || !buf || cap == 0) return ALLEGRO_E_INVALID;
  std::string out = "{\"graph_replays\": " + std::to_string(c->graph_replays) + ", \"graph_kernels\": " +
                    std::to_string(c->graph_launches) + ", \"current\": \"" + tune_name(c->tune) +
                    "\", \"buckets\": {";
  bool first = true;
  for (auto& kv : c->tuned) {
    out += std::string(first ? "" : ", ") + "\"" + kv.first + "\": {\"best\": \"" + tune_name(kv.second.best) +
           "\", \"trials\": {";
    first = false;
    for (size_t q = 0; q < kv.second.trials.size(); ++q) {
      char line[160];
      snprintf(line, sizeof line, "%s\"%s#%zu\": %.4f", q ? ", " : "", kv.second.trials[q].first.c_str(), q,
               kv.second.trials[q].second);
      out += line;
    }
    out += "}}";
  }
  out += "}}";
  if (out.size() + 1 > cap) return fail(c, ALLEGRO_E_CAPACITY, "report needs %zu bytes", out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return ALLEGRO_OK;
}

allegro_status allegro_set_md_skin(allegro_ctx* c, double skin) {
  if (!c) return ALLEGRO_E_INVALID;
  if (!(skin >= 0.0) || !std::isfinite(skin) || skin > 4.0 * c->arch.rc)
    return fail(c, ALLEGRO_E_INVALID, "md skin %g outside [0, 4 r_c]", skin);
  c->md_skin = skin;
  return ALLEGRO_OK;
}

allegro_status allegro_md_rebuilds(const allegro_ctx* c, int64_t* rebuilds) {
  if (!c || !rebuilds) return ALLEGRO_E_INVALID;
  *rebuilds = c->md_rebuilds;
  return ALLEGRO_OK;
}

allegro_status allegro_list_size(const allegro_ctx* c, int64_t* n_atoms, int64_t* n_edges, int32_t* n_struct) {
  if (!c) return ALLEGRO_E_INVALID;
  if (n_atoms) *n_atoms = c->have_nb ? c->n_atoms : 0;
  if (n_edges) *n_edges = c->have_nb ? c->n_edges : 0;
  if (n_struct) *n_struct = c->have_nb ? c->nstruct : 0;
  return ALLEGRO_OK;
}

allegro_status allegro_get_neighbors(allegro_ctx* c, int32_t* i, int32_t* j, int32_t* shift, int64_t cap) {
  if (!c) return ALLEGRO_E_INVALID;
  if (!c->have_nb) return fail(c, ALLEGRO_E_STATE, "no neighbour list");
  if (cap < c->n_edges) return fail(c, ALLEGRO_E_CAPACITY, "cap %lld < %lld edges", (long long)cap, (long long)c->n_edges);
  cudaSetDevice(c->device);
  const size_t E = (size_t)c->n_edges;
  allegro_status s;
  if ((s = copy_out(c, i, c->d_ei, E * 4)) != ALLEGRO_OK) return s;
  if ((s = copy_out(c, j, c->d_ej, E * 4)) != ALLEGRO_OK) return s;
  if ((s = copy_out(c, shift, c->d_eS, E * 12)) != ALLEGRO_OK) return s;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return ALLEGRO_OK;
}

allegro_status allegro_profile(allegro_ctx* c, int32_t enable) {
  if (!c) return ALLEGRO_E_INVALID;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  c->prof.on = enable != 0;
  c->prof.recs.clear();
  return ALLEGRO_OK;
}

allegro_status allegro_profile_report(allegro_ctx* c, char* buf, size_t cap, int64_t* launches) {
  if (!c) return ALLEGRO_E_INVALID;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (launches) *launches = c->launches;
  if (!buf || cap == 0) return ALLEGRO_OK;
  struct Agg { int n = 0; double ms = 0, flops = 0, bytes = 0; };
  std::vector<std::pair<std::string, Agg>> agg;
  for (const ProfRec& r : c->prof.recs) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->prof.ev[2 * r.ev], c->prof.ev[2 * r.ev + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    Agg* a = nullptr;
    for (auto& p : agg)
      if (p.first == r.name) a = &p.second;
    if (!a) {
      agg.push_back({r.name, Agg()});
      a = &agg.back().second;
    }
    a->n += r.launches;
    a->ms += ms;
    a->flops += r.flops;
    a->bytes += r.bytes;
  }
  std::string out = "{";
  for (size_t q = 0; q < agg.size(); ++q) {
    char line[256];
    snprintf(line, sizeof line, "%s\"%s\": {\"launches\": %d, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
             q ? ", " : "", agg[q].first.c_str(), agg[q].second.n, agg[q].second.ms, agg[q].second.flops,
             agg[q].second.bytes);
    out += line;
  }
  out += "}";
  if (out.size() + 1 > cap) return fail(c, ALLEGRO_E_CAPACITY, "report needs %zu bytes", out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return ALLEGRO_OK;
}

const char* allegro_last_error(const allegro_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

void allegro_destroy(allegro_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
  for (void* p : c->weight_allocs) cudaFree(p);
  void* bufs[] = {c->d_map, c->d_pos, c->d_types, c->d_species, c->d_row_ptr, c->d_col_ptr, c->d_count,
                  c->d_cell_of, c->d_wrap, c->d_sorted, c->d_pos4, c->d_pw, c->d_atom_struct, c->d_Eatom, c->d_F, c->d_Wat,
                  c->d_ej, c->d_ei, c->d_eS, c->d_ed, c->d_col_edge, c->d_Ee, c->d_g, c->d_cell_count,
                  c->d_cell_start, c->d_cell_cursor, c->d_offs, c->d_cells, c->d_pbc, c->d_nimg, c->d_Eout,
                  c->d_Wout, c->d_scan_tmp, c->d_err, c->d_total, c->d_minmax, c->d_red_scratch, c->ws,
                  c->d_md_pos, c->d_md_vel, c->d_md_invm, c->d_md_types, c->d_md_masses, c->d_md_E, c->d_md_K,
                  c->d_md_part, c->d_pair_basis, c->d_pair_rc2, c->d_zbl, c->d_sk_row, c->d_sk_j,
                  c->d_sk_S, c->d_sk_ref, c->d_cell9, c->d_maxd, c->d_amax, c->d_wraps};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

}  // extern "C"
