/*
 * allegro.h -- C ABI of the GB300 (sm_103a) Allegro edge hot path.
 *
 * Computes, for a set of atoms, the strictly local Allegro potential of
 * arXiv 2304.10061: ordered neighbour pairs within r_c, Bessel x envelope
 * radial basis, real spherical harmonics, the two-body MLP, per layer the
 * env-weight projection, the environment sum and the Clebsch-Gordan tensor
 * product (Eq. 1), the latent MLP, then the edge-energy MLP, the float64
 * per-atom scale/shift/sum (Sec. "Allegro", "Mixed-precision calculations"),
 * and, through a hand-written adjoint, forces F = -dE/dpos and the virial.
 *
 * Conventions for every entry point:
 *   - Every call returns an allegro_status; no exception crosses the ABI.
 *     On failure allegro_last_error(ctx) holds a one-line description.
 *   - Input and output arrays are owned by the caller.  Each may live in host
 *     memory or in device memory of the context's GPU; the library detects
 *     which (cudaPointerGetAttributes) and copies as needed.  Host inputs are
 *     copied before the call returns; host outputs are complete when it
 *     returns.  Device outputs are complete when work queued on the
 *     context's stream (allegro_set_stream) has finished; calls themselves
 *     synchronise that stream before returning.
 *   - Units: Angstrom, eV, eV/Angstrom.  All outputs are float64.
 *   - A context is not thread safe; use one per host thread.
 */
#ifndef ALLEGRO_H
#define ALLEGRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct allegro_ctx allegro_ctx;

typedef enum {
  ALLEGRO_OK = 0,
  ALLEGRO_E_INVALID = 1,    /* bad argument: null pointer, bad size, unknown type, non-finite input, bad weights */
  ALLEGRO_E_OOM = 2,        /* device memory could not be allocated */
  ALLEGRO_E_CUDA = 3,       /* a CUDA runtime call failed */
  ALLEGRO_E_CAPACITY = 4,   /* more edges than allegro_reserve(..., fixed=1) allows; last_error gives the need */
  ALLEGRO_E_TIMEOUT = 5,    /* a bounded device-side wait ran out (kernel returned early, results invalid) */
  ALLEGRO_E_NONFINITE = 6,  /* an output is NaN or Inf */
  ALLEGRO_E_STATE = 7       /* call out of order (e.g. energy_forces before neighbors) */
} allegro_status;

typedef enum {
  ALLEGRO_PREC_FP32 = 0,    /* all MLP GEMMs in float32 on the CUDA cores */
  ALLEGRO_PREC_BF16 = 1,    /* MLP GEMMs in bfloat16 on tcgen05 tensor cores, float32 accumulation */
  ALLEGRO_PREC_TF32 = 2,    /* float32 weights and activations, MLP GEMMs read as TF32 by tcgen05
                               (kind::tf32), float32 accumulation: Table IV's production setting */
  ALLEGRO_PREC_FP8 = 3      /* MLP GEMMs with E4M3 operands on tcgen05 (kind::f8f6f4), float32
                               accumulation; per-tensor power-of-two scales: each weight matrix's
                               fixed at allegro_create (max|W| maps to <= 448), each activation's
                               from the max|value| its producer recorded in the same evaluation
                               (max maps to <= 224); activations stored in bfloat16 (converted to
                               E4M3 on chip).  Sec. "Mixed-precision calculations" taken one
                               step below bfloat16: forces carry E4M3 rounding (3 mantissa bits),
                               an error of order 10% of RMS|F| on the seeded models; for
                               precision studies, not for MD */
} allegro_precision;

/*
 * allegro_create -- load a model and bind a context to one GPU.
 *   weights_blob/blob_bytes: host memory, an "ALGW" v1 weights image (header
 *       with the architecture, then float32 weights and float64 per-species
 *       scale sigma_Z / shift mu_Z of Sec. "Allegro": E = sum_i sigma_Z E_i + mu_Z).
 *       Copied; the caller may free it after the call.
 *   species_map[n_types]: maps the caller's atom type t to a model species
 *       (0..n_species-1).  NULL means the identity (types are species).
 *   r_c: neighbour cutoff in Angstrom; <= 0 takes the model's cutoff, any
 *       other value must equal it (the radial basis and envelope vanish there).
 *   precision: an allegro_precision.
 *   device: CUDA device ordinal.  out: receives the context.
 * Supported models: 1 to 3 layers, l_max 1 to 3 (three-layer models carry
 * pseudo-parity features in their middle layers), channels a power of two from
 * 8 to 128, MLP widths up to 1024 (the paper's production model: two-body
 * [128, 256, 512, 1024], latent 3 x 1024; with the BF16 path, MLPs wider than
 * 256 need channels x (l_max + 1) a multiple of 64).  Others return
 * ALLEGRO_E_INVALID.
 */
allegro_status allegro_create(const void* weights_blob, size_t blob_bytes,
                              const int32_t* species_map, int32_t n_types,
                              double r_c, int32_t precision, int32_t device,
                              allegro_ctx** out);

/* allegro_set_stream -- queue all later device work on `cuda_stream` (a
 * cudaStream_t of the context's device; NULL = the context's own stream). */
allegro_status allegro_set_stream(allegro_ctx* ctx, void* cuda_stream);

/*
 * allegro_reserve -- pre-size the device arena for `atom_cap` atoms and
 * `edge_cap` ordered edges (the role of the paper's 5 % input padding,
 * Sec. "Optimized LAMMPS-Kokkos implementation": no reallocation while sizes
 * fluctuate).  fixed = 0: later calls still grow the arena when needed (with
 * 5 % headroom).  fixed = 1: a neighbour build needing more edges fails with
 * ALLEGRO_E_CAPACITY and last_error states the required count.
 * chunk_edges > 0 caps the edges evaluated per pass of the model (the
 * activation working set scales with it); 0 = automatic.
 */
allegro_status allegro_reserve(allegro_ctx* ctx, int64_t atom_cap, int64_t edge_cap,
                               int32_t fixed, int64_t chunk_edges);

/*
 * allegro_set_pair_cutoffs -- per-ordered-species-pair cutoffs (Sec.
 * "Species-dependent cutoffs"): edge (i, j) exists iff |d|^2 < rc^2 with
 * rc = pair_rc[Z_i * n_species + Z_j] (row = the centre atom's model species,
 * column = the neighbour's), and its Bessel basis and envelope use that rc
 * (B_n(r) = sqrt(2/rc) sin(n pi r / rc) / r, u(r / rc)).
 *   pair_rc: host memory, n_species x n_species float64, every entry in
 *       (0, r_c] of the model; NULL restores the model cutoff for every pair.
 *   n_species: must equal the model's species count.
 * The neighbour list must be rebuilt afterwards (energy_forces returns
 * ALLEGRO_E_STATE until then).  allegro_neighbors_noalloc ignores the table.
 * Errors: ALLEGRO_E_INVALID (bad count or entry), ALLEGRO_E_CUDA.
 */
allegro_status allegro_set_pair_cutoffs(allegro_ctx* ctx, const double* pair_rc, int32_t n_species);

/*
 * allegro_set_zbl -- add the ZBL screened nuclear repulsion (Sec. "Training
 * details": the production potential carries a ZBL term) to every energy
 * evaluation:  per ordered edge (i, j), half of
 *   E_ZBL(r) = k_e Z_a Z_b / r * phi(r / a_s) * u(r / rc),
 *   a_s = 0.8854 a_0 / (Z_a^0.23 + Z_b^0.23),  k_e = 14.399645 eV A,  a_0 = 0.529177 A,
 *   phi(x) = 0.18175 e^-3.19980x + 0.50986 e^-0.94229x + 0.28022 e^-0.40290x + 0.02817 e^-0.20162x
 * (the universal ZBL screening function), u the model's envelope with the
 * edge's cutoff, is added to atom i's energy after the per-species scale and
 * shift (E_i = sigma_Z E_i^model + mu_Z + sum_j E_ZBL(r_ij) / 2), with its
 * forces and virial.  Evaluated in float32 per edge, summed in float64.
 *   atomic_numbers: host, n_species int32 in 1..118 (Z of each model species);
 *       NULL removes the term.
 * Errors: ALLEGRO_E_INVALID (bad count or entry), ALLEGRO_E_CUDA.
 */
allegro_status allegro_set_zbl(allegro_ctx* ctx, const int32_t* atomic_numbers, int32_t n_species);

/*
 * allegro_neighbors -- build the ordered neighbour list of one structure.
 * An edge is (i, j, S), S in Z^3 an image shift, displacement
 *   d = (pos_j + (S0 a + S1 b) + S2 c) - pos_i  evaluated in float64 in that
 * order without fused multiply-add, kept iff |d|^2 < r_c^2 and not
 * (i == j and S == 0) (Sec. "Allegro": per-ordered-pair energies E_ij).
 *   n_atoms >= 0; pos[n_atoms*3] float64 (x,y,z per atom, any position, not
 *   necessarily inside the cell); types[n_atoms] int32 caller types;
 *   cell[9] float64 row-major with rows a, b, c, or NULL for no cell;
 *   pbc[3] (0/1 per axis; NULL = all periodic if cell given, else none).
 *   A periodic axis needs a cell.  n_edges_out (host, may be NULL): edges.
 * The result is kept in the context for allegro_energy_forces.
 */
allegro_status allegro_neighbors(allegro_ctx* ctx, int64_t n_atoms, const double* pos,
                                 const int32_t* types, const double* cell, const uint8_t* pbc,
                                 int64_t* n_edges_out);

/*
 * allegro_neighbors_local -- the neighbour list of one sub-domain of a spatial
 * decomposition (Sec. "Optimized LAMMPS-Kokkos implementation": strict
 * locality lets each rank evaluate its own atoms with a ghost halo of width
 * r_c).  Atoms [0, n_local) are the sub-domain's own atoms and the only
 * centres; atoms [n_local, n_atoms) are ghosts (copies of other sub-domains'
 * atoms, already shifted by the periodic image they stand for), which appear
 * only as neighbours j.  Same pair rule and arguments as allegro_neighbors.
 * allegro_energy_forces then returns E_total = the sum of the local atoms'
 * energies, E_atom = 0 for ghosts, F for every atom (a ghost's force is its
 * share of the local energies, to be added to the atom it copies), and the
 * virial of the local centres' edges.  Summed over sub-domains whose local
 * atoms partition the system and whose ghosts cover r_c around them, these
 * equal the single-domain results.
 */
allegro_status allegro_neighbors_local(allegro_ctx* ctx, int64_t n_local, int64_t n_atoms, const double* pos,
                                       const int32_t* types, const double* cell, const uint8_t* pbc,
                                       int64_t* n_edges_out);

/*
 * allegro_neighbors_batched -- many independent structures in one packed
 * list.  Structure b holds atoms [atom_offsets[b], atom_offsets[b+1]);
 * atom_offsets[n_struct+1] int64 (host or device).  cells[n_struct*9] or
 * NULL (no cells); pbc[n_struct*3] or NULL (periodic iff a cell is given).
 * No edge joins two structures.  Intended for many small structures
 * (each evaluated by all-pairs search over its image range).
 */
allegro_status allegro_neighbors_batched(allegro_ctx* ctx, int32_t n_struct,
                                         const int64_t* atom_offsets, const double* pos,
                                         const int32_t* types, const double* cells,
                                         const uint8_t* pbc, int64_t* n_edges_out);

/*
 * allegro_energy_forces -- evaluate the model on the last neighbour list.
 *   E_total: [1] (single structure) or [n_struct] (batched), per-structure
 *            sum of sigma_Z E_i + mu_Z, float64.  Required.
 *   E_atom:  [n_atoms] sigma_Z E_i + mu_Z or NULL.
 *   F:       [n_atoms*3] forces -dE/dpos or NULL.
 *   virial:  [9] or [n_struct*9] row-major W_ab = -sum_e d_{e,a} dE/dd_{e,b}, or NULL.
 * The adjoint runs when F or virial is requested.
 */
allegro_status allegro_energy_forces(allegro_ctx* ctx, double* E_total, double* E_atom,
                                     double* F, double* virial);

/*
 * allegro_md_verlet -- velocity-Verlet molecular dynamics of one structure
 * (Sec. "Problem Overview": MD integrates Newton's equations with femtosecond
 * time steps): per step v += dt/2 F/m, x += dt v, neighbour rebuild, forces,
 * v += dt/2 F/m, all on the GPU.
 *   pos[n_atoms*3] (A) and vel[n_atoms*3] (A/fs): in/out, host or device.
 *   types[n_atoms]: caller types (mapped as in allegro_neighbors);
 *   masses[n_types]: amu per caller type (host or device), all > 0.
 *   cell, pbc: as allegro_neighbors (positions are not wrapped).
 *   dt: fs; n_steps >= 0.  E_pot, E_kin: [n_steps+1] (eV) or NULL, the
 *   potential (sum sigma_Z E_i + mu_Z) and kinetic energy at steps 0..n_steps.
 * Forces and the neighbour list of the final positions stay in the context.
 */
allegro_status allegro_md_verlet(allegro_ctx* ctx, int64_t n_atoms, double* pos, double* vel,
                                 const int32_t* types, const double* masses, int32_t n_types,
                                 const double* cell, const uint8_t* pbc, double dt, int64_t n_steps,
                                 double* E_pot, double* E_kin);

/*
 * allegro_set_md_skin -- neighbour reuse with a Verlet skin in
 * allegro_md_verlet (the paper's MD runs keep neighbour lists between
 * rebuilds, Sec. "Results"): skin > 0 builds a candidate list at r_c + skin
 * and rebuilds it only once some atom has moved skin/2 since; every step the
 * exact list (the same pair rule as allegro_neighbors) is filtered from the
 * candidates, so energies and forces are those of a rebuild every step.
 * skin = 0 (the default) rebuilds every step.  skin in [0, 4 r_c], finite.
 * allegro_md_rebuilds -- candidate-list builds (or full rebuilds when the
 * skin is 0) made by the last allegro_md_verlet call, into *rebuilds.
 */
allegro_status allegro_set_md_skin(allegro_ctx* ctx, double skin);
allegro_status allegro_md_rebuilds(const allegro_ctx* ctx, int64_t* rebuilds);

/*
 * allegro_list_size -- atoms, edges and structures of the neighbour list the
 * context holds (the last allegro_neighbors*, or the final positions of
 * allegro_md_verlet); zeros when it holds none.  Any output may be NULL.
 */
allegro_status allegro_list_size(const allegro_ctx* ctx, int64_t* n_atoms, int64_t* n_edges, int32_t* n_struct);

/*
 * allegro_get_neighbors -- copy the last neighbour list out, sorted by centre
 * atom i (rows in ascending i; order inside a row is deterministic but
 * unspecified).  i[cap], j[cap], shift[cap*3] int32 (any may be NULL);
 * cap must be >= the edge count.
 */
allegro_status allegro_get_neighbors(allegro_ctx* ctx, int32_t* i, int32_t* j, int32_t* shift,
                                     int64_t cap);

/*
 * allegro_set_autotune -- enable (1) or disable (0) the launch-configuration
 * autotuner (Sec. "Optimized LAMMPS-Kokkos implementation": the workload's
 * shapes fluctuate; the configuration is picked per shape).  When enabled,
 * the first allegro_energy_forces of each shape bucket (edges and atoms at
 * quarter-octave resolution, energy-only or with forces, single or batched)
 * times candidate configurations by coordinate descent -- edges per chunk
 * (the largest that fits, 1/2, 1/4, 1/8 of the list), each fused MLP layer
 * pair on or off, epilogue warps per TMEM quarter of the arithmetic GEMM
 * epilogues -- and keeps the fastest for that bucket (the first call takes
 * about a dozen evaluations).  Every candidate computes the same function.
 * Disabling restores the defaults.  An allegro_reserve chunk size overrides
 * the tuned one.
 *
 * allegro_set_graphs -- enable (1) or disable (0) replay of the evaluation as
 * a CUDA graph: the device work of allegro_energy_forces (all chunks, the
 * MLP GEMMs, row kernels and reductions) is captured the second time the same
 * shape, chunking, buffer addresses, configuration and stream are seen, and
 * replayed with one cudaGraphLaunch while they stay the same (a changed edge
 * count or a reallocation falls back to eager launches and recaptures).
 * Ignored while allegro_profile is on.
 *
 * allegro_autotune_report -- JSON into buf[cap] (host): the current
 * configuration, graph replays and kernels per graph, and per tuned bucket
 * the chosen configuration and every trial's time in ms.
 * ALLEGRO_E_CAPACITY if cap is too small.
 */
allegro_status allegro_set_autotune(allegro_ctx* ctx, int32_t enable);
allegro_status allegro_set_graphs(allegro_ctx* ctx, int32_t enable);
allegro_status allegro_autotune_report(allegro_ctx* ctx, char* buf, size_t cap);

/*
 * allegro_profile -- enable (1) or disable (0) per-launch timing of the
 * library's kernels with CUDA events on the context's stream; enabling clears
 * earlier records.  Not part of the method: a tracing aid.
 * allegro_profile_report -- writes a JSON object into buf[cap] (host):
 *   {"<kernel>": {"launches": n, "ms": total, "flops": algorithmic FLOPs,
 *                 "bytes": algorithmic bytes}, ...}
 * over the launches recorded since profiling was enabled, and the number of
 * kernel launches this context has issued since creation into *launches
 * (may be NULL).  ALLEGRO_E_CAPACITY if cap is too small.
 */
allegro_status allegro_profile(allegro_ctx* ctx, int32_t enable);
allegro_status allegro_profile_report(allegro_ctx* ctx, char* buf, size_t cap, int64_t* launches);

/*
 * allegro_neighbors_noalloc -- the ordered neighbour list of one small
 * structure, computed without allocating any device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory while they run (an MD engine whose memory pool owns the GPU, a
 * loop that must keep a fixed footprint), and so cannot create a context.
 * Same pair rule as allegro_neighbors (exact float64 test of every candidate
 * image, strict r < r_c), by an all-pairs search (meant for small structures).
 *   pos[n_atoms*3]: device float64, any positions (not necessarily wrapped
 *       into the cell); n_atoms <= 16384 (larger sizes return
 *       ALLEGRO_E_CAPACITY: the scratch is a fixed device array of about
 *       128 KiB).  A non-finite position, or two positions more than 1e8 cell
 *       widths apart, returns ALLEGRO_E_INVALID.
 *   cell[9] (rows a, b, c) and pbc[3]: HOST pointers or NULL (no cell: no
 *       periodicity; pbc NULL: every axis periodic).  r_c > 0 and finite, and
 *       r_c <= 4 perpendicular cell widths along each periodic axis, else
 *       ALLEGRO_E_INVALID.  Inputs needing more than 6e10 (pair, image)
 *       candidate tests return ALLEGRO_E_CAPACITY before any launch.
 *   i[cap], j[cap], shift[cap*3]: device int32 outputs, rows in ascending i.
 *       *n_edges (host): the edge count; ALLEGRO_E_CAPACITY if it exceeds cap
 *       or INT32_MAX (outputs then untouched).
 *   stream: cudaStream_t (NULL = legacy default stream).  The call reads the
 *       edge count back to the host between its two passes and synchronises
 *       the stream before it returns.
 * Runs on the current device.  Its scratch array lives in the library on every
 * device that loads it, until process exit.  The first call on a device looks
 * up the array's address there; make it before any stream capture.  Calls
 * share the array: calls that overlap on the GPU race and corrupt results.
 */
allegro_status allegro_neighbors_noalloc(const double* pos, int64_t n_atoms, const double* cell,
                                         const uint8_t* pbc, double r_c, int32_t* i, int32_t* j,
                                         int32_t* shift, int64_t cap, int64_t* n_edges, void* stream);

/* allegro_last_error -- description of the last failure on ctx (never NULL). */
const char* allegro_last_error(const allegro_ctx* ctx);

/* allegro_destroy -- free the context and its device memory (NULL is a no-op). */
void allegro_destroy(allegro_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ALLEGRO_H */
