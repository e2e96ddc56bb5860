// Internal declarations shared by the translation units of liballegro_gb300.
// Host orchestration lives in context.cu; kernels in neighbors.cu,
// edge_kernels.cu, row_kernels.cu, gemm_simt.cu and gemm_tc.cu.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/allegro.h"

namespace alg {

typedef __nv_bfloat16 bf16;

// Largest sizes the kernels are instantiated for.
constexpr int kMaxLmax = 3;
constexpr int kMaxS = (kMaxLmax + 1) * (kMaxLmax + 1);   // spherical-harmonic components
constexpr int kMaxChannels = 128;
constexpr int kMaxWidth = 1024;
constexpr int kMaxSpecies = 64;
constexpr int kMaxBessel = 16;

// Device error word bits (set by kernels, read by the host after each call).
enum DevErr : int {
  kErrTimeout = 1,      // a bounded mbarrier wait ran out
  kErrNeighbor = 2,     // neighbour fill pass disagreed with its count pass
  kErrBadInput = 4,     // non-finite coordinates or an unknown type
  kErrNonFinite = 8,    // a per-atom energy or force is NaN / Inf
};

struct Arch {
  int ns = 0, nb = 0, p = 0, lmax = 0, nl = 0, C = 0;
  double rc = 0, ann = 0;
  // per-ordered-species-pair cutoffs (Sec. "Species-dependent cutoffs"), set by
  // allegro_set_pair_cutoffs: device [ns * ns][2] = {1/rc, sqrt(2/rc)} of pair
  // (Z_i, Z_j) for the basis and envelope, and device [ns * ns] rc^2 for the
  // neighbour test; null: the model cutoff rc for every pair
  const float* pair_basis = nullptr;
  const double* pair_rc2 = nullptr;
  // ZBL repulsion (Sec. "Training details"), set by allegro_set_zbl: device
  // [ns * ns][2] = {k_e Z_a Z_b / 2, 1 / a_s} per ordered species pair; null: no ZBL term
  const float* zbl = nullptr;
  std::vector<int> tb, lat, edge;
  // evaluated through the generic row path (three layers, l_max 3, or the FP8 precision)
  bool generic = false;
  int S() const { return (lmax + 1) * (lmax + 1); }
  int n_w() const { return C * (lmax + 1); }
  int K0in() const { return 2 * ns + nb; }
  int Klat(int L) const { return L == 0 ? tb.back() : lat.back(); }
};

// A linear map W [N x K] (out x in) with the device copies the GEMMs use:
// forward B = W ([N][ld] row-major), backward B = W^T ([K][ldT]).
struct Lin {
  int N = 0, K = 0, ld = 0, ldT = 0;
  float* f32 = nullptr;
  float* f32T = nullptr;
  bf16* b16 = nullptr;
  bf16* b16T = nullptr;
  // FP8 precision: E4M3 copies [N][ld8] and [K][ld8T] (pitches multiples of 16 bytes) with their
  // per-tensor power-of-two scales (W = s8 q8)
  uint8_t* f8 = nullptr;
  uint8_t* f8T = nullptr;
  int ld8 = 0, ld8T = 0;
  float s8 = 1.0f, s8T = 1.0f;
};

// Tensor-product constants of one model, passed to kernels by value.
struct TPConst {
  float W1[kMaxS * kMaxS * kMaxS];  // fused path tensor of layer 1 (when 2 layers): W[a][b][c]
  float clast[kMaxS];               // last layer: s = sum_a clast[a] V_a Gamma_a (diagonal of W[a][b][0])
  float nu;                         // environment normalisation 1/sqrt(avg_num_neighbors)
};

// Nonzero pattern of the fused path tensor W[a][b][c] of a layer whose inputs
// and outputs are natural-parity irreps, l_max <= 2, real spherical harmonics
// ordered m = -l..l within each l (index a = l^2 + l + m).  W[a][b][c] can be
// nonzero only if (l_a, l_b, l_c) satisfies the triangle rule with l_a + l_b +
// l_c even (parity), |m_c| = |m_a| + |m_b| or ||m_a| - |m_b|| (the product of
// two real harmonics carries only those |m|), and the sine/cosine type of m_c
// (m < 0: sine) is the product of the types of m_a and m_b (sin sin and cos cos
// give cos, sin cos gives sin).  The host checks every loaded tensor against it.
__host__ __device__ constexpr int sh_l(int a) { return a < 1 ? 0 : (a < 4 ? 1 : (a < 9 ? 2 : 3)); }
__host__ __device__ constexpr int sh_m(int a) { return a - sh_l(a) * sh_l(a) - sh_l(a); }
__host__ __device__ constexpr int iabs_c(int x) { return x < 0 ? -x : x; }
__host__ __device__ constexpr bool tp_nonzero(int a, int b, int c) {
  return iabs_c(sh_l(a) - sh_l(b)) <= sh_l(c) && sh_l(c) <= sh_l(a) + sh_l(b) &&
         ((sh_l(a) + sh_l(b) + sh_l(c)) & 1) == 0 &&
         (iabs_c(sh_m(c)) == iabs_c(sh_m(a)) + iabs_c(sh_m(b)) ||
          iabs_c(sh_m(c)) == iabs_c(iabs_c(sh_m(a)) - iabs_c(sh_m(b)))) &&
         ((sh_m(c) < 0) == ((sh_m(a) < 0) != (sh_m(b) < 0)));
}
// some c with W[a][b][c] possibly nonzero
__host__ __device__ constexpr bool tp_any_c(int a, int b, int S) {
  bool r = false;
  for (int c = 0; c < S; ++c) r = r || tp_nonzero(a, b, c);
  return r;
}

enum Epi : int {
  EPI_FWD_SILU = 0,   // pre = acc (optional store); out = silu(acc) * (rowscale ? rowscale[m] : 1)
  EPI_F32 = 1,        // out(f32) = acc + (add ? add[m][n] : 0)
  EPI_BWD_SILU = 2,   // out = acc * silu'(pre[m][n])
  // Adjoint head of x = u * silu(z) fused into the GEMM producing xbar
  // (BF16 path, whole rows per CTA): xbar = acc + add; out = xbar u silu'(z);
  // ubar[m] += sum_n xbar_n silu(z_n).
  EPI_HEAD = 3,
  // Last latent layer fused with the folded edge-energy MLP and the start of
  // the adjoint (BF16 path, whole rows per CTA): z = acc, h = silu(z);
  // E[m] = u sum_n v_n h_n;  ubar[m] = sigma_m sum_n v_n h_n;
  // out = sigma_m v u silu'(z)  (the gradient w.r.t. z, input of the adjoint GEMMs).
  EPI_LAST = 4,
  EPI_LINEAR = 5,     // out = acc in the activation type (bf16 on the BF16 path)
};

struct GemmArgs {
  const char* label = "gemm";      // profiling label
  int M = 0, N = 0, K = 0;
  const void* A = nullptr; int lda = 0;     // [M][lda] activations (float or bf16)
  // tcgen05 path only: columns [K1, K) of A taken from a second array A2 ([M][lda2], bf16);
  // K1 a multiple of 64 (the operand k-block)
  const void* A2 = nullptr; int lda2 = 0; int K1 = 0;
  const Lin* W = nullptr; bool trans = false;
  const bf16* Bover = nullptr; int ldb_over = 0;   // tcgen05 path: B [N][ld] given directly (W unused)
  int b_row0 = 0;                                  // tcgen05 path: first row of B (W's matrix) used
  int epi = EPI_F32;
  void* out = nullptr; int ldo = 0;
  void* pre = nullptr; int ldp = 0;
  const float* rowscale = nullptr;
  // addend [M][ld_add]: float for EPI_F32, the activation type (bf16) for EPI_HEAD on the BF16 path
  const void* add = nullptr; int ld_add = 0;
  float* ubar = nullptr;           // EPI_HEAD / EPI_LAST
  const float* v = nullptr;        // EPI_LAST: folded edge-energy vector [N]
  const float* rowsig = nullptr;   // EPI_LAST: sigma_{Z_i} per row
  float* Eout = nullptr;           // EPI_LAST: E_ij per row
  int epq = 4;                     // tcgen05 path: epilogue warps per TMEM quarter of SiLU-adjoint / last-layer GEMMs
  // FP8 path: B given directly as E4M3 [N][ld] with its scale (the K-concatenated head maps)
  const uint8_t* Bover8 = nullptr; int ldb_over8 = 0; float sBover8 = 1.0f;
  // FP8 path: per-tensor amax slots (float bits, device) of A, of A2, and of this GEMM's output
  const unsigned* amax_a = nullptr;
  const unsigned* amax_a2 = nullptr;
  unsigned* amax_out = nullptr;
};

// ---- launchers -----------------------------------------------------------
// GEMMs
void gemm_simt_f32(const GemmArgs& g, cudaStream_t st);
bool gemm_tc_bf16(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why);
bool gemm_tc_init(std::string* why);
// float32 operands read as TF32 by tcgen05 kind::tf32, float32 epilogues (FWD_SILU, F32, BWD_SILU, LINEAR)
bool gemm_tc_tf32(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why);
bool gemm_chain_bf16(const GemmArgs& g1, const GemmArgs& g2, cudaStream_t st, int* d_err, std::string* why);
// E4M3 operands with per-tensor scales read by tcgen05 kind::f8f6f4 (bf16 activations converted on
// chip), float32 accumulation, bf16 / float32 epilogues (FWD_SILU, F32, BWD_SILU, LINEAR)
bool gemm_tc_fp8(const GemmArgs& g, cudaStream_t st, int* d_err, std::string* why);
// dst[r][k] = e4m3(src[r][k] * inv_scale) for k < cols, 0 for cols <= k < ldd (rows x ldd bytes)
void fp8_quantize(const float* src, int rows, int cols, int lds, uint8_t* dst, int ldd, float inv_scale,
                  cudaStream_t st);

// scan / utilities
void exclusive_scan_i32(const int* in, int* out, int n, int* d_total, void* tmp, size_t tmp_bytes,
                        cudaStream_t st);
size_t scan_tmp_bytes(int n);

// neighbours
struct CellGrid {
  double inv[9];      // inverse cell (row-major), frac = pos * inv (row vector times matrix)
  double cell[9];
  int pbc[3];
  int n[3];           // cells per axis
  int R[3];           // stencil radius per axis
  double lo[3], span[3];   // non-periodic axes: frac range mapped onto the grid
  int n_centres;      // atoms [0, n_centres) are centres; the rest (ghosts) only neighbours
};
void nb_bin(const double* pos, int n, const CellGrid& g, int* cell_of, int* wrap, int* cell_count,
            cudaStream_t st);
void nb_place(const int* cell_of, int n, const int* cell_start, int* cell_cursor, int* sorted,
              cudaStream_t st);
void nb_sort_cells(const int* cell_start, int n_cells, int* sorted, cudaStream_t st);
// pos4[s].w carries the model species of atom sorted[s] (its bits)
// pos4 / pw / wraps: wrapped float32 (with the species bits) and float64 positions and the
// wrap counts, all in cell order
void nb_pos4(const double* pos, const int* species, int n, const CellGrid& g, const int* wrap, const int* sorted,
             float4* pos4, double* pw, int4* wraps, cudaStream_t st);
// pair_rc2: null, or device [ns * ns] squared cutoffs per ordered species pair
// (each <= rc2, the search radius; `band` is the prefilter band of rc2)
void nb_search(bool fill, const double* pos, int n, const CellGrid& g, const int* cell_of,
               const int4* wraps, const int* cell_start, const int* sorted, const float4* pos4, const double* pw,
               double rc2, float band, const double* pair_rc2, int ns, int* count, const int* row_ptr, int* ej,
               int* ei, int* eS, double* ed, int* d_err, cudaStream_t st);
void nb_bruteforce_batched(bool fill, const double* pos, const int64_t* offs, int nstruct,
                           const double* cells, const int* pbc, const int* nimg, double rc2,
                           const int* species, const double* pair_rc2, int ns,
                           const int* atom_struct, int n, int* count, const int* row_ptr, int* ej,
                           int* ei, int* eS, double* ed, int* d_err, cudaStream_t st);
// Verlet-skin reuse: count (fill = false, into count[i]) or write (fill = true, rows at row_ptr[i]) the
// candidates of a list built at r_c + skin (sk_row / sk_j / sk_S) that pass the exact rule now
void nb_skin_filter(bool fill, const double* pos, int n, const double* d_cell, const int* sk_row, const int* sk_j,
                    const int* sk_S, double rc2, const double* pair_rc2, const int* species, int ns, int* count,
                    const int* row_ptr, int* ej, int* ei, int* eS, double* ed, cudaStream_t st);
// max_i |pos_i - ref_i|^2 as the bits of a double in *out (cleared first)
void nb_max_disp2(const double* pos, const double* ref, int n, unsigned long long* out, cudaStream_t st);
void nb_columns(const int* ej, int E, int n, int* col_count, cudaStream_t st);
void nb_fill_columns(const int* ej, int E, const int* col_ptr, int* cursor, int* col_edge,
                     cudaStream_t st);
void nb_sort_columns(const int* col_ptr, int n, int* col_edge, cudaStream_t st);
void nb_struct_span(const double* pos, const int64_t* offs, const double* inv, int nstruct, double* span,
                    cudaStream_t st);
void nb_minmax_frac(const double* pos, int n, const double* inv, double* d_minmax, cudaStream_t st);

// edge kernels
// geometry, basis (Y, u, sigma_{Z_i}) and the first two-body layer (pre-activation Z0, activation H0,
// times u when that layer is the two-body MLP's last); W0t = W0 transposed, [K0in][ldW] float32
template <typename T>
void edge_geom_fwd(int Ec, int e0, const double* ed, const int* ei, const int* ej, const int* species,
                   const Arch& a, float* Y, float* u, const double* sigma, float* sig, const float* W0t, int ldW,
                   T* Z0, int ldZ, T* H0, int ldH, bool scale_u, cudaStream_t st, unsigned* amax = nullptr);
// Partial adjoints of Y [Ec][S] written by the row-kernel passes
struct YbarParts {
  const float* p[2];
};
// edge forces g_ij from zbar0 (adjoint of the first two-body pre-activation), ubar and Ybar
template <typename T>
void edge_geom_bwd(int Ec, int e0, const double* ed, const int* ei, const int* ej, const int* species,
                   const Arch& a, const T* zbar0, int ldz, const float* W0t, int ldW, const float* ubar,
                   const YbarParts& yb, float* g, cudaStream_t st);
// (addx, if given: an activation-type addend of xbar, [Ec][ld_addx])
template <typename T>
void mlp_head_bwd(int Ec, int K, const float* xbar, int ld_x, const float* vconst, const int* ei,
                  const int* species, const double* sigma, int e0, const T* pre, int ld_pre, const float* u,
                  float* ubar, bool ubar_init, T* zbar, int ld_z, cudaStream_t st, unsigned* amax = nullptr,
                  const T* addx = nullptr, int ld_addx = 0);
template <typename T>
void edge_energy(int Ec, int K, const T* x, int ldx, const float* v, float* Ee, cudaStream_t st);
// float64 per-atom energies sigma_Z E_i + mu_Z (+ the ZBL term when a.zbl is set), forces by row and
// column gathers of dE/dd, per-atom virial
// atoms [n_centres, n) are ghosts: energy 0 (their own environments are incomplete); forces from the
// column gather (their share of the local centres' energies)
void atom_reduce(int n, int n_centres, const int* row_ptr, const int* col_ptr, const int* col_edge, const float* Ee,
                 const float* g, const double* ed, const int* species, const double* sigma, const double* mu,
                 bool want_forces, double* E_atom, double* F, double* Wat, const int* ei, const int* ej,
                 const Arch& a, cudaStream_t st);
void struct_reduce(int nstruct, const int64_t* offs, const double* E_atom, const double* Wat, const double* F,
                   bool want_w, double* E_out, double* W_out, int* d_err, double* scratch, int64_t n_atoms,
                   cudaStream_t st);

// velocity Verlet
void md_inv_mass(int n, const int* types, const double* masses, int nm, double* inv_m, int* err, cudaStream_t st);
void md_kick(int n, double* pos, double* vel, const double* F, const double* inv_m, double dt, bool drift,
             cudaStream_t st);
void md_kinetic(int n, const double* vel, const double* inv_m, double* part, double* out, cudaStream_t st);

// row (per-atom) kernels: environment sums and tensor products
struct RowIO {
  int a0 = 0, na = 0, e0 = 0;
  const int* row_ptr = nullptr;
  int C = 0;
  const float* Y = nullptr;            // [Ec][S]
  const void* W01 = nullptr; int ld01 = 0;    // w0 at column 0, w1 at column n_w (activation type)
  const void* w2 = nullptr; int ld2 = 0;      // (activation type)
  float* G1 = nullptr; float* G2 = nullptr;   // [na][C][S]
  void* xs = nullptr; int ldxs = 0; int xs_off = 0;   // s output (T), column offset
  const void* sbar1 = nullptr; const void* sbar2 = nullptr; int ld_sbar1 = 0, ld_sbar2 = 0;   // T
  void* wbar01 = nullptr; int ld_wbar01 = 0;  // T
  void* wbar2 = nullptr; int ld_wbar2 = 0;    // T
  // partial adjoints of Y, [Ec][S] each, written (not accumulated) by one pass each:
  //   one layer:  row_bwd_last pass 1 -> Ybar[0], pass 2 -> Ybar[1]
  //   two layers: row_bwd_last -> Ybar[0], row_bwd_mid (second pass) -> Ybar[1]
  float* Ybar[2] = {nullptr, nullptr};
};
// ---- any number of layers (row_generic.cu) ----
constexpr int kGenMaxLayers = 3;
// FP8 precision: amax slots per context (one per activation written in a chunk)
constexpr int kAmaxSlots = 128;
constexpr int kGenMaxD = 32;       // components of the largest feature (l_max 3, both parities: 31)
struct GenRowIO {
  int a0 = 0, na = 0, e0 = 0, C = 0, S = 0, lmax = 0, nl = 0;
  const int* row_ptr = nullptr;
  const float* Y = nullptr;                       // [Ec][S]
  float nu = 1.0f;
  // index L = 0 (embedding w^0) .. nl (env weights w^L): activation-type arrays, columns
  // [col, col + C (l_max+1)) of rows `ld` apart
  const void* w[kGenMaxLayers + 1] = {};
  int ldw[kGenMaxLayers + 1] = {}, wcol[kGenMaxLayers + 1] = {};
  void* wbar[kGenMaxLayers + 1] = {};
  int ldwbar[kGenMaxLayers + 1] = {}, wbcol[kGenMaxLayers + 1] = {};
  // L = 1..nl: s^L output (latent input's s columns) and its adjoint sbar^L
  void* xs[kGenMaxLayers + 1] = {};
  int ldxs[kGenMaxLayers + 1] = {}, xs_off[kGenMaxLayers + 1] = {};
  const void* sbar[kGenMaxLayers + 1] = {};
  int ldsbar[kGenMaxLayers + 1] = {}, sbar_off[kGenMaxLayers + 1] = {};
  // L = 1..nl, per atom [na][C][S]: Gamma^L (nu applied), Q^L, Gammabar^L
  float* G[kGenMaxLayers + 1] = {};
  float* Q[kGenMaxLayers + 1] = {};
  float* Gb[kGenMaxLayers + 1] = {};
  float* Qb = nullptr;                            // [na][C][S] scratch
  float* Ybar = nullptr;                          // [Ec][S]
  // layer tensors W^k, k = 1..nl: their values (host memory) at the candidate nonzeros that
  // gen_pack_values lists, layers 1..nl concatenated; the kernels take them as launch parameters
  const float* vals = nullptr;
  int dim[kGenMaxLayers + 1] = {};                // dim[0] = S, dim[nl] = 1
  // FP8 precision: amax slots (float bits) of the s columns written by the forward pass
  // and of the wbar arrays written by the adjoint pass (null: not recorded)
  unsigned* amax_s = nullptr;
  unsigned* amax_wbar = nullptr;
};
struct Irrep;
// The values of the layer tensors W[k] (k = 1..nl, dense float64 over dim(irs[k-1]) x S x
// dim(irs[k])) at the generic kernels' candidate nonzeros, in their order; false (with the
// reason) when the model is outside the generic kernels' set or a nonzero lies outside the
// candidates.
bool gen_pack_values(int lmax, int nl, const std::vector<std::vector<Irrep>>& irs,
                     const std::vector<std::vector<double>>& W, std::vector<float>& vals, std::string& why);
// forward of layer L: Gamma^L, Q^L, s^L
template <typename T>
void gen_row_fwd(const GenRowIO& io, int L, cudaStream_t st);
// adjoint of layer L (call for L = nl down to 1): Qbar^L, Gammabar^k (k <= L), wbar^L, w^0bar, Ybar
template <typename T>
void gen_row_bwd(const GenRowIO& io, int L, cudaStream_t st);

template <typename T>
void row_fwd(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st);
template <typename T>
void row_bwd(int layer, int nl, int lmax, const RowIO& io, const TPConst& tp, cudaStream_t st);

// host-side O(3) constants (independent implementation)
double cg_racah(int j1, int m1, int j2, int m2, int j3, int m3);
void coupling_real(int l1, int l2, int l3, std::vector<double>& out);   // [(2l1+1)(2l2+1)(2l3+1)]
void fused_layer_tensor(int lmax, const float* theta_raw, std::vector<double>& W, int& n_in, int& n_out,
                        bool last);
// any number of layers: irreps (l, p = +1 / -1) of V^0..V^nl, and the fused tensor of one layer
struct Irrep {
  int l, p;
};
void layer_irreps(int lmax, int nl, std::vector<std::vector<Irrep>>& irs);
int irreps_dim(const std::vector<Irrep>& v);
void layer_tensor(int lmax, const std::vector<Irrep>& in, const std::vector<Irrep>& out, const float* theta_raw,
                  std::vector<double>& W);

}  // namespace alg
