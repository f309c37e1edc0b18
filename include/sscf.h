/*
 * libsscf: sparse SCF hot path (Scemama, Renon & Rapacioli 2014, "A Sparse
 * SCF algorithm and its parallel implementation: Application to DFTB") on one
 * GB300 GPU (sm_103a).
 *
 * One context holds one water-like cluster: molecules of three consecutive
 * atoms (O, H, H), 6 atomic orbitals each (O s, px, py, pz, H s, H s), 4
 * doubly occupied and 2 virtual MOs per molecule. All device memory is owned
 * by the context; every host pointer passed in is read (or written) during
 * the call only and stays owned by the caller. Calls on one context run in
 * order on the context's CUDA stream and are not thread-safe.
 *
 * Status codes: every function returns SSCF_OK (0) or a negative error; no
 * exception or abort crosses this interface. Units: bohr, hartree, electrons.
 */
#ifndef SSCF_H
#define SSCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SSCF_OK = 0,
    SSCF_ERR_INVALID_ARG = -1,   /* bad pointer, size or value                      */
    SSCF_ERR_OOM = -2,           /* device allocation failed                         */
    SSCF_ERR_CUDA = -3,          /* a CUDA runtime call or a kernel launch failed    */
    SSCF_ERR_NONFINITE = -4,     /* NaN or Inf in an input or a result               */
    SSCF_ERR_CAPACITY = -5,      /* a sparse row outgrew its capacity; state kept    */
    SSCF_ERR_NOT_CONVERGED = -6, /* sscf_run reached max_scc; state kept             */
    SSCF_ERR_TIMEOUT = -7,       /* a bounded device wait gave up                    */
    SSCF_ERR_STATE = -8          /* call made out of order (e.g. step before guess)  */
};

enum { SSCF_FP64 = 0, SSCF_MIXED = 1 };
enum { SSCF_ORTHO_ALL = 0, SSCF_ORTHO_OCC = 1 };

typedef struct sscf_ctx sscf_ctx;

/* Geometry and partition (host arrays, copied at sscf_create). One context
 * may hold several independent clusters (batch mode): molecules of a cluster
 * are consecutive, clusters are numbered 0, 1, ... in order, groups never
 * span two clusters and are numbered cluster by cluster. Nothing couples two
 * clusters: no Hamiltonian or overlap element, no group neighbour, no gamma
 * term; every kernel launch serves all clusters at once. */
typedef struct {
    int n_atoms;              /* 3 * n_mol                                              */
    const int* species;       /* n_atoms: 0 = O, 1 = H; molecule-major O, H, H          */
    const double* xyz;        /* 3 * n_atoms, bohr                                       */
    const int* group_of_mol;  /* n_atoms / 3: MO-group index of every molecule (<= 8 per group) */
    const int* cluster_of_mol; /* n_atoms / 3: cluster index, or NULL for one cluster    */
} sscf_system;

/* Model and SCF parameters (Section "Specific implementation for DFTB",
 * Section "Sparsity and numerical accuracy"). */
typedef struct {
    double onsite[3];        /* O s, O p, H s on-site energies of H0                    */
    double V0[4];            /* H0 two-centre prefactors: ss-sigma, sp-sigma, pp-sigma, pp-pi */
    double S0[4];            /* overlap prefactors, same order                           */
    double r_decay;          /* V(r) = V0 exp(-r / r_decay)                              */
    double r_cut;            /* pairs with r <= r_cut interact                           */
    double U[2];             /* Hubbard parameters O, H: gamma = 1/sqrt(r^2 + a^2)       */
    double q0[2];            /* reference populations O, H                               */
    double eps;              /* sparse threshold epsilon of the current stage            */
    double dq_tol;           /* delta q_max convergence criterion                        */
    double e_tol;            /* |E_n - E_{n-1}| convergence criterion                    */
    double group_cut;        /* MO groups closer than this are neighbours (20 bohr)      */
    double rot_cap_factor;   /* at most factor * N_occ rotations per sweep (10)          */
    double mix_beta;         /* linear charge mixing                                     */
    int max_scc;             /* iteration limit of sscf_run (per stage)                  */
    int precision;           /* SSCF_FP64 or SSCF_MIXED                                   */
    int ortho_every;         /* 1: one occupied orthonormalisation pass per SCC step     */
    int cap_tiles;           /* per-row tile capacity of C; 0 picks the dense size       */
    int cap_y;               /* row blocks per tile of Y = X C; 0 picks the largest cluster */
    int apply_variant;       /* 0: specialised sweep kernels where a block allows them,
                                1: the generic kernel for every block,
                                2: the specialised kernels with one CTA per block
                                (all three give the same results; 1 and 2 are for tests) */
    int closure_mode;        /* structural fill of a sweep (same results either way):
                                0: once per sweep, every row given every tile its
                                   units are connected to through the sweep's active
                                   blocks (fewest launches; rows can grow to the whole
                                   cluster, so cap_tiles defaults to that);
                                k >= 1: once per window of k colours, a row given the
                                   tiles its units are connected to through the active
                                   blocks of those colours, counting only the units it
                                   holds nonzero values in; zero tiles are dropped at
                                   the end of the sweep. Rows hold their real fill plus
                                   one window's insertions (k = 1: the partner of each
                                   unit), for clusters whose dense rows do not fit; a
                                   larger k copies C fewer times but, with many active
                                   blocks, links units across much of the cluster
                                   within the window (k = 1 bounds it). With k >= 1 a
                                   CAPACITY error leaves the MOs partly swept: restart
                                   from a checkpoint. */
} sscf_params;

typedef struct {
    double energy;           /* E = sum P*H0 + 1/2 dq^T gamma dq (Ha)                    */
    double dq_max;           /* max_a |q_a^(n) - q_a^(n-1)|                               */
    double dE;               /* E^(n) - E^(n-1)                                          */
    double max_fov;          /* largest |F_ij| over kept occupied-virtual blocks          */
    double eta;              /* largest normalised off-diagonal overlap of the ortho pass */
    int64_t n_rot;           /* rotations applied in the sweep                           */
    int64_t n_combo;         /* orthonormalisation combinations applied                  */
    int64_t nnz_c;           /* stored values of C: tiles x 96 (6 AO rows x 16 MOs)       */
    int64_t nnz_occ;         /* stored values of the occupied tiles                      */
    int64_t launches;        /* kernels launched by the step                              */
    int64_t upd_rot;         /* 2x2 row updates applied by the rotation sweep (pairs x rows) */
    int64_t upd_combo;       /* 2x2 row updates applied by the orthonormalisation pass    */
    int iteration;
} sscf_step_info;

/* Grouping ----------------------------------------------------------------- */

/* MO groups for any geometry: constrained k-means of the molecules (Section
 * "Defining neighbouring lists of atoms and MOs"), run on the GPU. Every
 * molecule is one unit, placed at its first (oxygen) atom. Centres start on a
 * grid over the bounding box with at least ceil(n_mol / n_link) points (the
 * axis with the largest spacing refined first, extents below 1 bohr counted as
 * 1 bohr, points at lo + (2i + 1) L / 2g). Each iteration links every molecule
 * to a centre, at most n_link per centre: molecules propose to centres in
 * increasing (distance^2, centre index) and a centre keeps the n_link
 * proposals with the smallest (distance^2, molecule index) (deferred
 * acceptance; the result does not depend on any processing order, so the
 * paper's shuffle of the centres is not needed). Then every centre with
 * members moves to their centroid (summed in increasing molecule index),
 * until the average move of the centres is below tol (bohr) or after max_iter
 * iterations; the links of the last centres are returned. Groups are the
 * centres holding molecules, numbered in centre order.
 *   n_atoms, xyz: as sscf_system (host; molecules O, H, H)
 *   n_link: 1 .. 8 molecules per group
 *   group_of_mol: host, n_atoms / 3, written; n_groups_out, iters_out may be NULL
 * Device memory comes from the allocator of sscf_set_allocator, if set, and is
 * freed before the call returns. Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
int sscf_group_molecules(int n_atoms, const double* xyz, int n_link, int max_iter, double tol,
                         void* cuda_stream, int* group_of_mol, int* n_groups_out, int* iters_out);

/* Context ---------------------------------------------------------------- */

/* Builds the structure of step I (atom and molecule neighbour lists within
 * r_cut, the MO-group neighbour map at group_cut, the greedy colouring of the
 * group graph; Section "Defining neighbouring lists"), uploads the geometry,
 * evaluates H0 and S on the molecule-pair blocks and allocates C.
 * `cuda_stream` is a cudaStream_t or NULL for the legacy default stream.
 * Errors: INVALID_ARG (non-water layout, bad sizes), OOM, CUDA, NONFINITE. */
int sscf_create(const sscf_system* sys, const sscf_params* prm, void* cuda_stream,
                sscf_ctx** out);
void sscf_destroy(sscf_ctx* ctx);
const char* sscf_strerror(int status);

/* Device allocator used by the next sscf_create (NULL restores cudaMalloc /
 * cudaFree). alloc returns NULL on failure, which sscf_create reports as
 * SSCF_ERR_OOM. */
typedef void* (*sscf_alloc_fn)(size_t bytes, void* user);
typedef void (*sscf_free_fn)(void* ptr, void* user);
int sscf_set_allocator(sscf_alloc_fn alloc, sscf_free_fn free_, void* user);

/* Thresholds of the current SCF stage (Section "Sparsity and numerical
 * accuracy": loose eps 1e-3 / dq 1e-1, then the user values). */
int sscf_set_thresholds(sscf_ctx* ctx, double eps, double dq_tol, double e_tol);

/* Sizes: n_ao, n_mo, n_occ, n_groups, n_tiles, n_colours (any may be NULL). */
int sscf_get_dims(const sscf_ctx* ctx, int* n_ao, int* n_mo, int* n_occ, int* n_groups,
                  int* n_tiles, int* n_colours);

/* Steps ---------------------------------------------------------------- */

/* Step II (Section "Initial guess"): one non-SCC generalised eigensolve per
 * molecule; occupied MOs group-major, then virtual MOs; in a molecule the
 * MOs follow ascending eigenvalue, the largest-magnitude coefficient made
 * positive (first index within 1e-9 of the largest magnitude). */
int sscf_guess(sscf_ctx* ctx);

/* Step III (Section "Orthonormalization", steps a-e): passes of
 * sigma = C^T S C on neighbouring-group blocks, normalisation by diag(sigma),
 * first-order combinations C'_i = C_i - sigma_ij C_j / 2,
 * C'_j = C_j - sigma_ij C_i / 2 on pairs |sigma_ij| >= 1e-3 eta, truncation
 * at 1e-3 eps, until eta < target or max_pass passes. The target is eps / 100
 * (Section "Sparsity and numerical accuracy") floored at what the storage
 * resolves: max(eps / 100, 2^-19) (32 units in the last place of FP32) in
 * mixed precision, max(eps / 100, 1e-13) in FP64. The same target applies to
 * the occupied pass of every sscf_step. `which` is SSCF_ORTHO_ALL or
 * SSCF_ORTHO_OCC. passes_out, eta_out may be NULL. */
int sscf_orthonormalise(sscf_ctx* ctx, int which, int max_pass, int* passes_out,
                        double* eta_out);

/* Step IV, Eq. (H_dftb2): Q = gamma dq_in (all atom pairs, unscreened) is
 * kept from the last charge update; H = H0 + 1/2 S (Q_a + Q_b) on the
 * molecule-pair blocks, off-diagonal |H_mn| < eps set to zero. */
int sscf_build_fock(sscf_ctx* ctx);

/* A Fock (or any symmetric one-electron) matrix X built by the caller, for
 * methods whose step IV is not the DFTB build (Section "Algorithm and
 * computational details": only step IV is method specific; Section
 * "Computation kernel for the matrix products C^T X C"). X is given as dense
 * 6x6 blocks (row-major) on the molecule-pair pattern, in the pair order of
 * sscf_get_blocks (host, n_mp * 36 doubles); block (n, m) must be the
 * transpose of block (m, n). Off-diagonal |X_mn| < eps are set to zero, as
 * in sscf_build_fock, and X replaces H until the next sscf_build_fock. Use it
 * with sscf_rotate_sweep, sscf_orthonormalise and sscf_get_density_blocks;
 * sscf_step and sscf_run build the DFTB H themselves. Errors: INVALID_ARG,
 * NONFINITE, CUDA. */
int sscf_set_fock_blocks(sscf_ctx* ctx, const double* X);

/* Density matrix P = 2 C_occ C_occ^T (Eq. pop) of the current MOs on the
 * molecule-pair pattern, the input of the caller's next Fock build: dense
 * 6x6 blocks (row-major) in the pair order of sscf_get_blocks, into P (host,
 * n_mp * 36 doubles), summed in FP64. Charges and mixing state are not
 * changed. Errors: INVALID_ARG, STATE (before sscf_guess), OOM (its device
 * buffer is allocated by the first call), CUDA. */
int sscf_get_density_blocks(sscf_ctx* ctx, double* P);

/* Step V (Section "Partial diagonalization"): F = C^T H C on the occupied-
 * virtual blocks of neighbouring groups plus diag(F); pairs with
 * |F_ij| >= eps, at most rot_cap_factor * N_occ of the largest (ties kept);
 * Jacobi angles p, t, c, s in FP64 from the F of the sweep start; rotations
 * C'_i = c C_i + s C_j, C'_j = -s C_i + c C_j applied block colour by block
 * colour, then by in-block colour (i_loc + j_loc) mod n, truncating
 * |C| < eps after each. Outputs may be NULL. */
int sscf_rotate_sweep(sscf_ctx* ctx, int64_t* n_rot_out, double* max_fov_out);

/* Eq. (pop) with P = 2 C_occ C_occ^T on the molecule-pair pattern: Mulliken
 * charges q (host, n_atoms, or NULL), E = sum P*H0 + 1/2 dq^T gamma dq with
 * gamma dq recomputed from these charges, and max |q - q_previous|. The new
 * charges become q_previous and the SCC input is mixed:
 * dq_in += beta (dq - dq_in), Q_in += beta (gamma dq - Q_in). */
int sscf_density(sscf_ctx* ctx, double* q_out, double* E_out, double* dq_max_out);

/* Charges of the current C without mixing: they become q_previous, and the
 * SCC input is set to them (dq_in = dq, Q_in = gamma dq). This is how an SCF
 * stage starts after the guess and the orthonormalisation. E_out may be NULL. */
int sscf_reset_charges(sscf_ctx* ctx, double* E_out);

/* One SCC iteration: build_fock, rotate_sweep, one occupied ortho pass
 * (ortho_every = 1), density and mixing. */
int sscf_step(sscf_ctx* ctx, sscf_step_info* info);

/* Launch-shape autotuner (no counterpart in the paper): on the current state
 * it builds H and Y = H C as a step would, times the occupied-virtual transform
 * (three launches after one warm-up, CUDA events on the context's stream) for
 * 1, 2, 4 and 8 CTAs sharing each occupied tile's pairs, each with two
 * register budgets of the kernel (uncut, or cut for four resident CTAs per
 * SM), and keeps the fastest for later steps. Results of later calls do not
 * depend on the choice (each pair is summed the same way). Drops a captured
 * CUDA graph. tf_split_out (host, may be NULL) receives the CTAs per tile plus
 * 16 if the cut register budget won. Errors: STATE before sscf_guess, CUDA. */
int sscf_autotune(sscf_ctx* ctx, int* tf_split_out);

/* CUDA graphs: when enabled, sscf_step captures its device work (all kernel
 * launches of one SCC iteration) into a graph at the first call and replays
 * it afterwards: one launch per iteration. The graph is rebuilt when eps
 * changes or the C buffers swapped parity (sscf_set_C_dense, sscf_guess).
 * sscf_run and sscf_run_from_current then run each SCC stage as one graph
 * launch: a conditional while node repeats one captured SCC iteration and a
 * one-block kernel that applies the stage's convergence test on the device
 * (every cluster's max |q - q_prev| and |E - E_prev|), so no host round trip
 * separates the iterations; it stops at convergence, at max_scc iterations or
 * when a kernel reports an error, with the same results as the host loop.
 * (A stage whose captured iteration would not end in the C buffer it starts
 * from, possible with closure_mode 1, runs the host loop instead.) Needs a
 * non-NULL stream (SSCF_ERR_INVALID_ARG otherwise); per-launcher profiling
 * does not see replayed launches. */
int sscf_enable_graph(sscf_ctx* ctx, int enable);

/* Loose stage (eps 1e-3, dq 1e-1), full orthonormalisation, user stage until
 * dq_max <= dq_tol and |dE| <= e_tol in every cluster, final occupied orthonormalisation to
 * eps / 100 and final charges and energy. In mixed precision the SCC stages
 * orthonormalise to max(eps / 100, 2^-19) (see sscf_orthonormalise); before
 * the final orthonormalisation the context is widened to FP64
 * (sscf_set_precision), so the final MOs, charges and energy are FP64 and the
 * context stays FP64 afterwards. Returns NOT_CONVERGED with the state kept
 * if max_scc is reached. */
int sscf_run(sscf_ctx* ctx, sscf_step_info* info);

/* The user stage of sscf_run from the MOs already in the context (a
 * checkpoint restored with sscf_set_C_tiles, for example the converged MOs of
 * a nearby geometry, Section "Summary and future work": the MOs of one
 * geometry are a good start for the next): full orthonormalisation at eps,
 * charges of those MOs as the SCC input, SCC iterations until dq_max <= dq_tol
 * and |dE| <= e_tol, the final occupied orthonormalisation (in FP64, as
 * sscf_run). Errors: STATE before any MOs were set, NOT_CONVERGED (state
 * kept), and those of the steps. */
int sscf_run_from_current(sscf_ctx* ctx, sscf_step_info* info);

/* Storage precision of a live context (no counterpart in the paper, whose
 * orthonormalisation is FP64 and C^T H C FP32 throughout): SSCF_FP64 widens
 * C, H and every per-step buffer to FP64, SSCF_MIXED rounds C to FP32. The MO
 * coefficients and charges are kept (C converted value by value, H rebuilt
 * from the current SCC input); the last transform's F and pair lists are
 * dropped, and a captured CUDA graph is rebuilt at the next step. New buffers
 * are allocated before the old ones are freed. Errors: INVALID_ARG, OOM (the
 * context is then unchanged), CUDA. */
int sscf_set_precision(sscf_ctx* ctx, int precision);

/* Adjoint (no counterpart in the paper, which computes energies only): the
 * gradient of E = sum P*H0 + 1/2 dq^T gamma dq at the current MOs, assumed
 * converged and orthonormal (F_ov = 0, C^T S C = I):
 *   dE = sum P*dH0 + sum (1/2 P*(Q_a+Q_b) - W)*dS + 1/2 dq^T dgamma dq,
 *   W = 1/2 P H P = 2 C_occ F_oo C_occ^T  (energy-weighted density),
 * through the derivatives of the Slater-Koster blocks and of gamma.
 * dE_dxyz: host, 3*n_atoms (Ha/bohr, atom-major x, y, z), or NULL.
 * dE_dparams: host, 8: dE/dV0[0..3], dE/dS0[0..3], or NULL.
 * The charges of the current MOs become the SCC input (as sscf_reset_charges). */
int sscf_gradients(sscf_ctx* ctx, double* dE_dxyz, double* dE_dparams);

/* Batch mode: per-cluster results of the last charge update (sscf_step,
 * sscf_density, sscf_reset_charges, sscf_run): energies and max |q - q_prev|.
 * Outputs are host arrays of n_clusters entries (n_clusters_out, if not NULL,
 * receives the count; any array may be NULL). */
int sscf_get_cluster_results(sscf_ctx* ctx, double* energy, double* dq_max, int* n_clusters_out);

/* Tracing --------------------------------------------------------------- */

/* Per-launcher device times: when enabled, every kernel launcher of the steps
 * above is bracketed by CUDA events on the context's stream. */
int sscf_profile(sscf_ctx* ctx, int enable);
/* Summed milliseconds and call counts per launcher name since the last read
 * (then reset). names receives max_entries * 32 bytes, NUL-terminated; any
 * output may be NULL; n_out receives the number of names. Synchronises the
 * context's stream. */
int sscf_profile_read(sscf_ctx* ctx, int max_entries, char* names, double* ms, int64_t* calls, int* n_out);

/* State access (checkpoint / restart and tests) -------------------------- */

/* Dense copies for small systems: C is n_ao x n_mo, row-major (C[mu*n_mo+i]). */
int sscf_get_C_dense(sscf_ctx* ctx, double* C);
int sscf_set_C_dense(sscf_ctx* ctx, const double* C);
/* Rows of C for large systems: the AO rows `rows` (n of them), dense over
 * all MOs, into out (host, n x n_mo, row-major). */
int sscf_get_C_rows(sscf_ctx* ctx, int n, const int* rows, double* out);
/* Checkpoint and restart of C in its stored form (Section "Sparse storage",
 * here padded by row block): for every row block r (one molecule, 6 AO rows)
 * nt[r] stored tiles with sorted tile ids, each tile 96 values laid out
 * [6 AO rows][16 MOs] (MO columns past the tile's last MO are zero). Tiles of
 * the occupied MOs of group g have ids group-major from 0, then the virtual
 * tiles; all arrays are host memory owned by the caller, values in FP64 for
 * both precisions (a mixed context rounds them to FP32 on restart).
 * sscf_get_C_tiles: nt (n_mol ints), tiles (n_stored ints, row block after
 *   row block), vals (96 * n_stored doubles); any may be NULL, n_stored (if not
 *   NULL) receives the count, so a first call with NULL arrays sizes them.
 * sscf_set_C_tiles: the same arrays. Errors: INVALID_ARG (unsorted or foreign
 *   tile ids, negative counts), CAPACITY (more tiles than cap_tiles), NONFINITE,
 *   OOM; on any of these the MOs are left unchanged. The arrays go to the device
 *   in one copy each (page-locked host memory makes it faster) through a staging
 *   buffer the context allocates at the first call and keeps, grown as needed. */
int sscf_get_C_tiles(sscf_ctx* ctx, int32_t* nt, int32_t* tiles, double* vals, int64_t* n_stored);
int sscf_set_C_tiles(sscf_ctx* ctx, const int32_t* nt, const int32_t* tiles, const double* vals);
/* Columns of C for large systems: the MOs `cols` (n of them), dense over all
 * AOs, into out (host, n_ao x n, row-major). */
int sscf_get_C_cols(sscf_ctx* ctx, int n, const int* cols, double* out);
/* Entries F_ov(i, j) of the last transform for occupied i and virtual j
 * (global MO indices), 0 outside the kept blocks. */
int sscf_get_F_entries(sscf_ctx* ctx, int n, const int* i_mo, const int* j_mo, double* out);
/* Molecule-pair blocks: pairs (m, n) into mn (2 * n_mp) and the 6x6 blocks
 * (row-major) of the current H, of H0 and of S into n_mp * 36 doubles each.
 * Any array may be NULL; n_mp_out receives the number of blocks. */
int sscf_get_blocks(sscf_ctx* ctx, int* mn, double* H, double* H0, double* S, int64_t* n_mp_out);
/* Dense n_ao x n_ao copies of the current H, of H0 and of S. */
int sscf_get_H_dense(sscf_ctx* ctx, double* H, double* H0, double* S);
/* Dense F_ov (n_occ x (n_mo - n_occ), zero off the kept blocks) and diag(F)
 * (n_mo) of the last transform. */
int sscf_get_F_dense(sscf_ctx* ctx, double* F_ov, double* F_diag);
/* sigma = C^T S C of the last orthonormalisation pass, before normalisation
 * (Section "Orthonormalization", step b), dense over the pass's MOs (n x n,
 * row-major, n = n_occ after an occupied pass, n_mo after a pass over all
 * MOs; global MO order), zero off the blocks of neighbouring groups; the
 * passes read entry (i, j) with i before j in pass order, and both halves
 * hold it. n_out (may be NULL) receives n; sigma may be NULL to size it.
 * Errors: STATE before the first orthonormalisation pass. */
int sscf_get_overlap_dense(sscf_ctx* ctx, double* sigma, int* n_out);
/* Charges: q_prev (last output charges), dq_in and Q_in (SCC input). */
int sscf_get_charges(sscf_ctx* ctx, double* q_prev, double* dq_in, double* Q_in);
int sscf_set_charges(sscf_ctx* ctx, const double* q_prev, const double* dq_in,
                     const double* Q_in);
/* Group colouring (n_groups x n_groups, -1 off the graph) for structure tests. */
int sscf_get_colouring(sscf_ctx* ctx, int* colour);
/* Last pair list (rotations after sscf_rotate_sweep or sscf_step's sweep;
 * combinations after an orthonormalisation pass): for every pair its block
 * colour, in-block colour, and MO indices (i, j), grouped by colour, then
 * in-block colour. Any output array may be NULL; capacity is in pairs and
 * n_out receives the full count. */
int sscf_get_pairs(sscf_ctx* ctx, int64_t capacity, int32_t* colour_out, int32_t* sub_out, int32_t* i_out,
                   int32_t* j_out, int64_t* n_out);

/* Allocation-free pair selection ------------------------------------------
 *
 * No counterpart in the paper: this entry point exists for callers that
 * cannot call cudaMalloc (code running inside another framework's memory
 * pool, under a device-memory budget fixed at start-up, or where the
 * allocator belongs to someone else). It applies the same rule as the pair
 * selection inside sscf_rotate_sweep to an array the caller owns:
 * keep[i] = 1 iff |f[i]| >= tau, f[i] != 0, and |f[i]| is among the k_max
 * largest such values (all values tied with the k_max-th largest are kept).
 *
 *   f       device, n doubles (for example the entries of the kept F_ov blocks)
 *   keep    device, n bytes, written (0 or 1)
 *   n_keep  host, number of kept entries, or NULL (then the call does not
 *           synchronise the stream)
 *   stream  cudaStream_t or NULL
 *
 * It allocates nothing: its working memory is one file-scope __device__
 * array of 16 MiB + 2304 bytes that every GPU loading the library holds
 * until the process exits. n above 2^21 (2,097,152) is rejected with
 * SSCF_ERR_INVALID_ARG. The first call on a device (with that device
 * current) looks up the array's device address, and so does the first call
 * after that device's context was reset (cudaDeviceReset); make those calls
 * before any stream capture. All calls share the array and it keeps the last call's
 * contents (each call clears what must start at zero); calls that overlap on
 * the GPU, from other streams or host threads, race on it. */
int sscf_select_pairs_noalloc(const double* f, int64_t n, double tau, int64_t k_max, unsigned char* keep,
                              int64_t* n_keep, void* stream);

#ifdef __cplusplus
}
#endif
#endif
