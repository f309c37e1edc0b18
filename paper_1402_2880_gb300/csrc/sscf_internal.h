// Internal state and kernel launchers of libsscf.
//
// Data layout in HBM (one context = one cluster):
//   * row block      = one molecule = 6 AO rows (O s, px, py, pz, H1 s, H2 s);
//   * tile           = 16 consecutive MOs of one group's occupied (or virtual)
//                      list; occupied tiles come first (group-major), then
//                      the virtual tiles;
//   * C (MO coefficients) is stored row-major by row block: row block r holds
//     c_nt[r] tiles, ids sorted ascending in c_tile[r*cap + s], values
//     c_val[((r*cap + s)*6 + k)*16 + col] for AO row k of the molecule. The
//     paper's list-of-lists columns padded to s_m (Section "Sparse storage")
//     become rows padded to `cap` tiles: rotations are row-local, so a row is
//     the unit that grows and shrinks.
//   * H0, S, H are stored as dense 6x6 blocks on the molecule-pair pattern
//     (any atom pair within r_cut), CSR over the first molecule.
//   * the column index of C lists, per tile, the row blocks holding it
//     (sorted) and the slot inside each row.
//   * Y = X C (X = H or S) is stored column-major by tile: y_row[t*capY+k],
//     values y_val[((t*capY + k)*6 + row)*16 + col].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sscf.h"

namespace sscf {

constexpr int kAoPerMol = 6;
constexpr int kTileW = 16;
constexpr int kTileVals = kAoPerMol * kTileW;  // 96
constexpr int kMaxMolPerGroup = 8;
constexpr int kMaxDynSmem = 227 * 1024;          // dynamic shared memory a CTA may opt into
constexpr int kMaxSub = 48;                    // in-block colours (<= MOs per group side)
constexpr int kRotCap = 32 * 16;               // pairs of one occupied-virtual block
constexpr int kOrthoCap = 48 * 48;             // pairs of one orthonormalisation block

// Error word bits set by kernels (read back by the host after a step).
enum : unsigned {
    kErrCapacity = 1u,       // a row of C or a column of Y ran out of slots
    kErrSortSize = 2u,       // a column segment exceeded the in-smem sort size
    kErrNonFinite = 4u,      // NaN / Inf produced
    kErrGuess = 8u,          // per-molecule eigensolve failed (S not positive definite)
};

struct DeviceScalars {
    unsigned err;
    unsigned long long cand;      // candidate rotation pairs |F| >= tau
    unsigned long long n_rot;     // rotations kept
    unsigned long long n_combo;   // ortho combinations kept
    unsigned long long thr_key;   // bit pattern of the smallest kept |F| (double)
    unsigned long long sel_prefix;
    unsigned long long sel_mask;
    unsigned long long sel_k;     // rank still to find inside the prefix
    double max_fov;               // bits via atomicMax on the double's pattern
    double eta;
    double e_band;
    double e_coul;
    double dq_max;
    double energy;
    unsigned long long tiles[2];  // stored tiles of C, occupied tiles among them
    unsigned long long upd[2];    // 2x2 row updates of the sweep: rotations, combinations
    unsigned long long hist[256];
};

struct Ctx {
    sscf_params prm;
    cudaStream_t stream = nullptr;
    int prec = SSCF_FP64;
    size_t tsize = 8;  // bytes of one stored C / H / Y value

    // sizes
    int n_atoms = 0, n_mol = 0, n_ao = 0, n_occ = 0, n_mo = 0;
    int n_groups = 0, n_tiles = 0, n_occ_tiles = 0, n_colours = 0;
    int n_mp = 0;        // molecule-pair blocks, including (m, m)
    int n_clusters = 1;
    int max_cl_mol = 0;       // molecules of the largest cluster
    int max_cl_otiles = 0;    // occupied tiles of the largest cluster
    int max_cl_tiles = 0;     // tiles of the largest cluster
    int n_gnb = 0;       // group-graph entries (directed, including (A, A))
    int cap = 0;         // tiles per row block of C
    int capY = 0;        // row blocks per tile of Y
    int closure_window = 0;  // colours per closure (bounded fill); 0: one closure per sweep
    int apply_variant = 0;   // 0 specialised sweep kernels where they apply, 1 generic only,
                             // 2 specialised with one CTA per block
    int tf_split = 4;        // CTAs sharing one occupied tile's pairs in the transform (sscf_autotune)
    int tf_regs = 0;         // transform register budget: 0 uncut, 1 cut for 4 CTAs per SM (sscf_autotune)
    int n_sm = 152;          // multiprocessors of the context's device
    bool have_guess = false;
    int iteration = 0;
    long long n_launch = 0;   // kernels launched by this context
    double e_prev = 0.0;
    bool have_e_prev = false;
    int last_sched_kind = 0;   // 0 none, 1 rotations, 2 combinations
    double ortho_tol = 0.0;    // target of the orthonormalisation pass being launched
    int last_ortho_which = 0;

    // host copies of the structure
    std::vector<int> h_species;
    std::vector<double> h_xyz;
    std::vector<int> h_mol_group, h_mol_local, h_mol_cluster;
    std::vector<int> h_cl_mol0, h_cl_nmol;    // molecule range of every cluster
    std::vector<int> h_cl_g0;                 // group range of every cluster (n_clusters + 1)
    int max_cl_groups = 0;
    std::vector<int> h_mp_ptr, h_mp_col;
    std::vector<int> h_group_nmol, h_group_occ0, h_group_virt0;
    std::vector<int> h_group_ot0, h_group_not, h_group_vt0, h_group_nvt;
    std::vector<int> h_tile_group, h_tile_kind, h_tile_loc0, h_tile_nmo, h_tile_mo0;
    std::vector<int> h_gnb_ptr, h_gnb_col, h_gnb_row, h_gnb_colour;
    std::vector<int> h_colour_ptr, h_colour_blk;        // all directed blocks by colour
    std::vector<int> h_ocolour_ptr, h_ocolour_blk;      // blocks with A <= B by colour
    std::vector<int> h_colour_nfull, h_ocolour_nfull;   // leading blocks of each colour between full groups
    // tile-pair lists of the transforms
    std::vector<int> h_rot_tp_ptr;   // per a-tile CSR into (b, out) for the F_ov blocks
    std::vector<int> h_rot_tp_b, h_rot_tp_out;
    std::vector<int> h_rot_blk_tp0;  // first tile pair of every directed block
    int n_rot_tp = 0;

    // device: geometry and model
    double* d_xyz = nullptr;
    int* d_species = nullptr;
    int* d_mp_ptr = nullptr;
    int* d_mp_col = nullptr;
    int* d_mp_rev = nullptr;          // n_mp: the entry of (n, m) for the entry of (m, n)
    double* d_dens_part = nullptr;    // n_mp x 4: a pair's share of q (3 atoms) and band energy for its first row
    int* d_mp_row = nullptr;
    double* d_H0b = nullptr;
    double* d_Sb = nullptr;
    void* d_Hb = nullptr;       // T
    void* d_Sbt = nullptr;      // S in T precision (for S C in mixed mode)

    // device: groups, tiles, group graph
    int* d_mol_group = nullptr;
    int* d_mol_local = nullptr;
    int* d_group_nmol = nullptr;
    int* d_group_ot0 = nullptr;
    int* d_group_not = nullptr;
    int* d_group_vt0 = nullptr;
    int* d_group_nvt = nullptr;
    int* d_group_occ0_mo = nullptr;   // global index of the group's first occupied MO
    int* d_group_virt0_mo = nullptr;  // global index of the group's first virtual MO
    int* d_self_blk = nullptr;        // group-graph entry of (g, g)
    std::vector<int> h_self_blk;
    int* d_tile_group = nullptr;
    int* d_tile_row0 = nullptr;       // first molecule of the tile's cluster
    int* d_mol_cluster = nullptr;
    int* d_mol_row0 = nullptr;        // first molecule of the molecule's cluster
    int* d_mol_ot0 = nullptr;         // first occupied tile of the molecule's cluster
    int* d_atom_lo = nullptr;         // atom range of the atom's cluster
    int* d_atom_hi = nullptr;
    int* d_cl_mol0 = nullptr;
    int* d_cl_g0 = nullptr;           // n_clusters + 1: first group of every cluster
    int* d_cl_ot0 = nullptr;          // n_clusters + 1: first occupied tile of every cluster
    int* d_cl_vt0 = nullptr;          // n_clusters + 1: first virtual tile of every cluster
    int* d_clblk_ptr[2] = {nullptr, nullptr};   // blocks of every cluster: [0] all directed, [1] A <= B
    int* d_clblk[2] = {nullptr, nullptr};
    int* d_unit_lab = nullptr;        // 2 n_groups: closure component labels (cluster-local)
    int* d_lab_start = nullptr;       // 2 n_groups each: members of every closure component (CSR by label)
    int* d_lab_cnt = nullptr;
    int* d_lab_mem = nullptr;
    int* d_cl_nmol = nullptr;
    int* d_group_cl = nullptr;        // cluster of every group
    void* d_cl_sel = nullptr;         // per-cluster top-k state (6 words each)
    std::vector<unsigned long long> h_cl_sel_init;
    unsigned long long* d_cl_sel_init = nullptr;   // initial per-cluster top-k state (device copy)
    unsigned long long* d_cl_hist = nullptr;   // per-cluster radix histograms (256 each)
    double* d_cl_eta = nullptr;       // per-cluster largest normalised overlap
    double* d_cl_E = nullptr;         // per-cluster energy of the last charge update
    double* d_cl_dq = nullptr;        // per-cluster max |q - q_prev|
    double* d_cl_Eprev = nullptr;     // per-cluster energy of the previous iteration (graph-resident stages)
    int* d_loop = nullptr;            // graph-resident stage: iterations, converged
    int* d_tile_kind = nullptr;
    int* d_tile_loc0 = nullptr;
    int* d_tile_nmo = nullptr;
    int* d_tile_mo0 = nullptr;
    int* d_gnb_ptr = nullptr;
    int* d_gnb_row = nullptr;
    int* d_gnb_col = nullptr;
    int* d_gnb_colour = nullptr;
    int* d_colour_ptr = nullptr;
    int* d_colour_blk = nullptr;
    int* d_ocolour_ptr = nullptr;
    int* d_ocolour_blk = nullptr;

    // device: C (two buffers), its column index
    int* d_c_nt[2] = {nullptr, nullptr};
    int* d_c_tile[2] = {nullptr, nullptr};
    void* d_c_val[2] = {nullptr, nullptr};
    unsigned char* d_c_nz[2] = {nullptr, nullptr};   // per (row block, slot): 0 = tile known all-zero during a sweep
    unsigned char* d_c_cnz = nullptr;   // the current sweep's flags in column-index order
    int* d_blk_info = nullptr;          // per block of a sweep in colour order: 8 ints the FP32 sweep kernel starts from
    int cur = 0;
    int* d_cci_ptr = nullptr;     // n_tiles + 1
    int* d_cci_cnt = nullptr;     // n_tiles
    int* d_cci_row = nullptr;     // n_mol * cap
    int* d_cci_slot = nullptr;

    // device: Y = X C column-major
    int* d_y_n = nullptr;         // n_tiles
    int* d_y_row = nullptr;       // n_tiles * capY
    void* d_y_val = nullptr;      // n_tiles * capY * 96

    // device: transform outputs
    int* d_rot_tp_ptr = nullptr;
    int* d_rot_tp_b = nullptr;
    int* d_rot_tp_out = nullptr;
    int* d_rot_blk_tp0 = nullptr;
    void* d_F = nullptr;          // n_rot_tp * 256 (T)
    int* d_diag_tp_ptr = nullptr; // identity lists for the diagonal tile pairs
    int* d_diag_tp_b = nullptr;
    int* d_diag_tp_out = nullptr;
    void* d_Fdiag_tiles = nullptr;   // n_tiles * 256 (T)
    double* d_Fd = nullptr;       // n_mo

    // device: orthonormalisation tile-pair lists
    int n_ort_tp[2] = {0, 0};     // [0] all MOs, [1] occupied only
    int* d_ort_tp_ptr[2] = {nullptr, nullptr};
    int* d_ort_tp_b[2] = {nullptr, nullptr};
    int* d_ort_tp_out[2] = {nullptr, nullptr};
    int* d_ort_blk_tp[2] = {nullptr, nullptr};   // per directed block: 3x3 tile-pair ids (-1 none)
    std::vector<int> h_ort_blk_tp[2];
    void* d_sig = nullptr;        // max(n_ort_tp) * 256 (T)
    double* d_scale = nullptr;    // n_mo: 1/sqrt(sigma_ii)

    // device: pair schedules (rotations and combinations share the storage)
    int* d_pr_n = nullptr;        // n_gnb
    int* d_pr_lvl = nullptr;      // n_gnb * (kMaxSub + 1)
    uint16_t* d_pr_ij = nullptr;  // n_gnb * kOrthoCap
    void* d_pr_cs = nullptr;      // n_gnb * kOrthoCap * 2 (T)
    int* d_pr_touch = nullptr;    // n_gnb: side tiles touched (bits 0-2 side A, 3-5 side B)

    // device: charges
    double* d_q = nullptr;        // n_atoms, new charges
    double* d_q_prev = nullptr;
    double* d_dq_in = nullptr;
    double* d_Q_in = nullptr;
    double* d_dq = nullptr;
    double* d_Q = nullptr;
    double* d_e_mol = nullptr;    // n_mol band-energy partials
    double* d_P = nullptr;        // n_mp * 36: density blocks (allocated by the first sscf_get_density_blocks)
    unsigned char* d_stage = nullptr;   // staging of sscf_set_C_tiles (grown as needed)
    size_t stage_bytes = 0;
    double* d_red = nullptr;      // reduction scratch (n_mol + 1024)
    double* d_grad = nullptr;     // 3 n_atoms: dE/dxyz
    double* d_par = nullptr;      // 8: dE/d(V0, S0)
    double* d_gmol = nullptr;     // 9 n_mol: per-molecule force partials
    double* d_pmol = nullptr;     // 8 n_mol: per-molecule parameter partials
    DeviceScalars* d_sc = nullptr;
    DeviceScalars* h_sc = nullptr;   // pinned mirror

    std::vector<void*> allocations;

    // CUDA graph of one SCC step (sscf_enable_graph)
    bool use_graph = false;
    bool graph_valid = false;
    int graph_cur = 0;
    long long graph_launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;

    // per-launcher CUDA-event timing (off by default)
    bool prof = false;
    struct ProfRec {
        int id;
        cudaEvent_t e0, e1;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<std::string> prof_names;
    std::vector<double> prof_ms;
    std::vector<long long> prof_calls;
};

// ---- memory -----------------------------------------------------------------
int dev_alloc(Ctx* c, void** p, size_t bytes);
void dev_release(Ctx* c, void* p);   // frees one allocation of dev_alloc
void* raw_alloc(size_t bytes);       // device memory outside a context (the allocator hook if set); NULL on failure
void raw_free(void* p);
void dev_free_all(Ctx* c);

template <typename P>
inline int dalloc(Ctx* c, P** p, size_t n) {
    return dev_alloc(c, reinterpret_cast<void**>(p), n * sizeof(P));
}

// ---- kernel launchers (defined in the .cu files) ------------------------------
// model
cudaError_t launch_sk_blocks(Ctx* c);
cudaError_t launch_gamma(Ctx* c, const double* dq, double* Q);
cudaError_t launch_build_h(Ctx* c, double eps_threshold);
cudaError_t launch_guess(Ctx* c);
// sparse structure and products
cudaError_t launch_colindex(Ctx* c);
// Y = X C for tiles [tile_lo, tile_hi) on the row blocks reachable from each
// tile's rows; tiles below own_below on their own rows only
cudaError_t launch_xc(Ctx* c, bool use_h, int tile_lo, int tile_hi, int own_below = 0);
// Y = H C for the transform of a sweep: virtual tiles on every reachable row
// block (F_ov), occupied tiles on their own rows (only their diagonal blocks)
cudaError_t launch_xc_rot(Ctx* c);
cudaError_t launch_transform_rot(Ctx* c);
cudaError_t launch_transform_ortho(Ctx* c, int which);
cudaError_t launch_density(Ctx* c, double* P_out = nullptr);   // P blocks (n_mp x 36) too, if not NULL
// schedules and sweeps
cudaError_t launch_select_rot(Ctx* c);
cudaError_t launch_ortho_prepare(Ctx* c, int which, double tol);
// structural fill of the sweep's colours [col_lo, col_hi) (col_hi < 0: all); cur <- other
cudaError_t launch_closure(Ctx* c, int mode, int which, int col_lo = 0, int col_hi = -1, bool first = true);
size_t closure_smem_bytes(const Ctx* c);
size_t closure_labels_smem_bytes(const Ctx* c);
// mode 0 rotations, 1 combinations, colours [col_lo, col_hi) (col_hi < 0: all); in place
cudaError_t launch_apply(Ctx* c, int mode, int which, int col_lo = 0, int col_hi = -1);
cudaError_t launch_compact(Ctx* c);                      // drop all-zero tiles; cur <- other
// charges
cudaError_t launch_charges_finish(Ctx* c, bool mix);
cudaError_t launch_count_tiles(Ctx* c, unsigned long long* out);
// adjoint
cudaError_t launch_adjoint(Ctx* c, double* d_grad, double* d_par, double* d_gmol, double* d_pmol);

}  // namespace sscf

struct sscf_ctx {
    sscf::Ctx c;
};
