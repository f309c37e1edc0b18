// Pair selection, block schedules and the row-local sweep (Section "Partial
// diagonalization" and Section "Orthonormalization", step d).
//
// The paper applies pair updates block-parallel: blocks of one label
// (Figure "jacobi") touch disjoint MOs and run concurrently, labels run one
// after the other. Here the labels are the colours of a greedy edge colouring
// of the MO-group graph, and inside a block pairs go by the in-block colour
// (i_loc + j_loc) mod n. Every 2x2 update uses coefficients fixed at the start
// of the sweep, so the whole sweep acts on each AO row of C independently:
// the apply kernel gives one CTA to one AO row, walks the colours in order
// and reads and writes C once.
#include <math.h>

#include <vector>

#include "sscf_internal.h"

#include <type_traits>

namespace sscf {

namespace {

__device__ __forceinline__ unsigned long long dkey(double v) { return (unsigned long long)__double_as_longlong(v); }

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
    atomicMax((unsigned long long*)addr, dkey(v));
}

// local MO index -> (side tile position, column) for a group side made of
// `no` occupied MOs (tiles first) and then virtual MOs
__device__ __forceinline__ void side_pos(int loc, int no, int not_, int& tpos, int& col) {
    if (loc < no) {
        tpos = loc >> 4;
        col = loc & 15;
    } else {
        int v = loc - no;
        tpos = not_ + (v >> 4);
        col = v & 15;
    }
}

// --------------------------------------------------------------------------
// rotation candidates: count |F_ij| >= tau (F_ij != 0) per cluster and the
// largest |F|. The cap of rot_cap_factor * N_occ is a per-cluster rule: every
// cluster of a batch selects exactly as it would alone.
// --------------------------------------------------------------------------
struct ClSel {
    unsigned long long cand, prefix, mask, rank, thr, kmax;
};

template <typename T>
__global__ void k_rot_stats(int n_gnb, const int* __restrict__ gnb_row, const int* __restrict__ gnb_col,
                            const int* __restrict__ group_nmol, const int* __restrict__ group_nvt,
                            const int* __restrict__ group_cl, const int* __restrict__ blk_tp0,
                            const T* __restrict__ F, double tau, DeviceScalars* sc, ClSel* cl) {
    const int e = blockIdx.x;
    const int A = gnb_row[e], B = gnb_col[e];
    const int no = 4 * group_nmol[A], nv = 2 * group_nmol[B], nvt = group_nvt[B];
    unsigned cnt = 0;
    double mx = 0.0;
    for (int p = threadIdx.x; p < no * nv; p += blockDim.x) {
        const int i = p / nv, j = p % nv;
        const int tp = blk_tp0[e] + (i >> 4) * nvt + (j >> 4);
        const double f = fabs((double)F[(size_t)tp * 256 + (i & 15) * 16 + (j & 15)]);
        mx = fmax(mx, f);
        if (f >= tau && f > 0.0) ++cnt;
    }
    for (int off = 16; off > 0; off >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(&cl[group_cl[A]].cand, (unsigned long long)cnt);
        atomic_max_pos(&sc->max_fov, mx);
    }
}

// one radix-select pass over the candidate keys (8 bits, most significant
// first) of every cluster whose candidates exceed its cap. A CTA takes a
// contiguous range of blocks (clusters are contiguous in block order) and
// counts in shared memory, adding its nonzero bins to the cluster's global
// histogram when the cluster changes and at the end: the early passes put
// most keys in a few bins, which global atomics per key would serialise on.
template <typename T>
__global__ void __launch_bounds__(256) k_rot_hist(int shift, int n_gnb, const int* __restrict__ gnb_row,
                                                  const int* __restrict__ gnb_col,
                                                  const int* __restrict__ group_nmol, const int* __restrict__ group_nvt,
                                                  const int* __restrict__ group_cl, const int* __restrict__ blk_tp0,
                                                  const T* __restrict__ F, double tau,
                                                  const ClSel* __restrict__ cl, unsigned long long* __restrict__ hist) {
    __shared__ unsigned s_h[256];
    const int per = (n_gnb + gridDim.x - 1) / gridDim.x;
    const int e_lo = blockIdx.x * per, e_hi = min(n_gnb, e_lo + per);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_h[i] = 0u;
    int cur = -1;   // cluster whose counts s_h holds (the same in every thread)
    auto flush = [&]() {
        __syncthreads();
        for (int i = threadIdx.x; i < 256; i += blockDim.x)
            if (s_h[i]) {
                atomicAdd(&hist[(size_t)cur * 256 + i], (unsigned long long)s_h[i]);
                s_h[i] = 0u;
            }
        __syncthreads();
    };
    __syncthreads();
    for (int e = e_lo; e < e_hi; ++e) {
        const int A = gnb_row[e], B = gnb_col[e];
        const int c = group_cl[A];
        if (c != cur) {
            if (cur >= 0) flush();
            cur = c;
        }
        const ClSel s = cl[c];
        if (s.cand <= s.kmax) continue;
        const int no = 4 * group_nmol[A], nv = 2 * group_nmol[B], nvt = group_nvt[B];
        for (int p = threadIdx.x; p < no * nv; p += blockDim.x) {
            const int i = p / nv, j = p % nv;
            const int tp = blk_tp0[e] + (i >> 4) * nvt + (j >> 4);
            const double f = fabs((double)F[(size_t)tp * 256 + (i & 15) * 16 + (j & 15)]);
            if (!(f >= tau && f > 0.0)) continue;
            const unsigned long long k = dkey(f);
            if ((k & s.mask) != s.prefix) continue;
            atomicAdd(&s_h[(k >> shift) & 255ull], 1u);
        }
    }
    if (cur >= 0) flush();
}

// one thread per cluster: pick the bin holding the kmax-th largest key
// (last_shift: the final pass; keys below it are zero for every candidate)
__global__ void k_rot_pick(int shift, int last_shift, int n_clusters, ClSel* cl, unsigned long long* hist) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_clusters) return;
    ClSel s = cl[c];
    unsigned long long* h = hist + (size_t)c * 256;
    if (s.cand > s.kmax) {
        if (shift == 56) s.rank = s.kmax;
        unsigned long long cum = 0;
        int b = 255;
        for (; b > 0; --b) {
            if (cum + h[b] >= s.rank) break;
            cum += h[b];
        }
        s.prefix |= (unsigned long long)b << shift;
        s.mask |= 255ull << shift;
        s.rank -= cum;
        for (int i = 0; i < 256; ++i) h[i] = 0ull;
    }
    if (shift == last_shift) s.thr = s.cand > s.kmax ? s.prefix : 0ull;
    cl[c] = s;
}

// per block: kept pairs sorted by (in-block colour, i_loc) with Jacobi angles
// p = (F_ii - F_jj) / (2 F_ij), t = 1/(p + sgn(p) sqrt(1 + p^2)),
// c = 1/sqrt(1 + t^2), s = t c in FP64 (sgn(0) = +1)
template <typename T>
__global__ void k_rot_lists(int n_gnb, const int* __restrict__ gnb_row, const int* __restrict__ gnb_col,
                            const int* __restrict__ group_nmol, const int* __restrict__ group_nvt,
                            const int* __restrict__ group_occ0_mo, const int* __restrict__ group_virt0_mo,
                            const int* __restrict__ group_cl, const int* __restrict__ blk_tp0,
                            const T* __restrict__ F, const double* __restrict__ Fd, double tau, DeviceScalars* sc,
                            const ClSel* __restrict__ cl, int* __restrict__ pr_n,
                            int* __restrict__ pr_lvl, uint16_t* __restrict__ pr_ij, T* __restrict__ pr_cs,
                            int* __restrict__ pr_touch) {
    __shared__ unsigned char keep[32 * 16];
    __shared__ int cnt[kMaxSub + 1];
    const int e = blockIdx.x;
    const int A = gnb_row[e], B = gnb_col[e];
    const int no = 4 * group_nmol[A], nv = 2 * group_nmol[B], nvt = group_nvt[B];
    const int nsub = max(no, nv);
    const unsigned long long thr = cl[group_cl[A]].thr;
    __shared__ int s_touch;
    if (threadIdx.x == 0) s_touch = 0;
    __syncthreads();
    int touch_t = 0;   // side tiles this thread's kept pairs touch: bits 0-2 side A, 3-5 side B
    for (int p = threadIdx.x; p < 32 * 16; p += blockDim.x) {
        int i = p >> 4, j = p & 15;
        unsigned char kp = 0;
        if (i < no && j < nv) {
            const int tp = blk_tp0[e] + (i >> 4) * nvt + (j >> 4);
            const double f = fabs((double)F[(size_t)tp * 256 + (i & 15) * 16 + (j & 15)]);
            kp = (f >= tau && f > 0.0 && dkey(f) >= thr) ? 1 : 0;
            if (kp) touch_t |= (1 << (i >> 4)) | (1 << (3 + (j >> 4)));
        }
        keep[p] = kp;
    }
    if (touch_t) atomicOr(&s_touch, touch_t);
    __syncthreads();
    if ((int)threadIdx.x < nsub) {
        const int s = threadIdx.x;
        int c = 0;
        for (int i = 0; i < no; ++i) {
            int j = ((s - i) % nsub + nsub) % nsub;
            if (j < nv && keep[i * 16 + j]) ++c;
        }
        cnt[s] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        int* lvl = pr_lvl + (size_t)e * (kMaxSub + 1);
        for (int s = 0; s < nsub; ++s) {
            lvl[s] = run;
            run += cnt[s];
        }
        for (int s = nsub; s <= kMaxSub; ++s) lvl[s] = run;
        pr_n[e] = run;
        cnt[kMaxSub] = run;
        if (run) atomicAdd(&sc->n_rot, (unsigned long long)run);
        pr_touch[e] = s_touch;
    }
    __syncthreads();
    if ((int)threadIdx.x < nsub) {
        const int s = threadIdx.x;
        int pos = pr_lvl[(size_t)e * (kMaxSub + 1) + s];
        for (int i = 0; i < no; ++i) {
            int j = ((s - i) % nsub + nsub) % nsub;
            if (!(j < nv && keep[i * 16 + j])) continue;
            const int tp = blk_tp0[e] + (i >> 4) * nvt + (j >> 4);
            const double fij = (double)F[(size_t)tp * 256 + (i & 15) * 16 + (j & 15)];
            const double fii = Fd[group_occ0_mo[A] + i], fjj = Fd[group_virt0_mo[B] + j];
            const double p = __ddiv_rn(__dsub_rn(fii, fjj), __dmul_rn(2.0, fij));
            const double sg = p >= 0.0 ? 1.0 : -1.0;
            const double t = __ddiv_rn(1.0, __dadd_rn(p, __dmul_rn(sg, sqrt(__dadd_rn(1.0, __dmul_rn(p, p))))));
            const double cc = __ddiv_rn(1.0, sqrt(__dadd_rn(1.0, __dmul_rn(t, t))));
            const double ss = __dmul_rn(t, cc);
            const size_t q = (size_t)e * kOrthoCap + pos;
            pr_ij[q] = (uint16_t)(i | (j << 8));
            pr_cs[2 * q] = (T)cc;
            pr_cs[2 * q + 1] = (T)ss;
            ++pos;
        }
    }
}

// --------------------------------------------------------------------------
// orthonormalisation: d_i = sqrt(sigma_ii), eta, pair lists
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_ortho_scale(int w, int t_lo, int t_hi, const int* __restrict__ tile_group,
                              const int* __restrict__ tile_kind, const int* __restrict__ tile_nmo,
                              const int* __restrict__ tile_mo0, const int* __restrict__ group_ot0,
                              const int* __restrict__ group_not, const int* __restrict__ group_vt0,
                              const int* __restrict__ self_blk, const int* __restrict__ blk_tp,
                              const T* __restrict__ sig, double* __restrict__ dsc, unsigned* err) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int t = t_lo + (idx >> 4), c = idx & 15;
    if (t >= t_hi) return;
    if (c >= tile_nmo[t]) return;
    const int g = tile_group[t];
    const int pos = tile_kind[t] == 0 ? t - group_ot0[g] : group_not[g] + (t - group_vt0[g]);
    const int tp = blk_tp[self_blk[g] * 9 + pos * 3 + pos];
    double s = (double)sig[(size_t)tp * 256 + c * 17];
    if (!(s > 0.0) || !isfinite(s)) {
        atomicOr(err, kErrNonFinite);
        s = 1.0;
    }
    dsc[tile_mo0[t] + c] = sqrt(s);
}

template <typename T>
__device__ __forceinline__ double sig_hat(const T* sig, const int* blk_tp, int e, bool same, int ia, int ib, int ci,
                                          int cj, double di, double dj) {
    int tp;
    double v;
    if (same && ib < ia) {
        tp = blk_tp[e * 9 + ib * 3 + ia];
        v = (double)sig[(size_t)tp * 256 + cj * 16 + ci];
    } else {
        tp = blk_tp[e * 9 + ia * 3 + ib];
        v = (double)sig[(size_t)tp * 256 + ci * 16 + cj];
    }
    return __ddiv_rn(v, __dmul_rn(di, dj));
}

// MO of local index `loc` in group g for the pass (occupied first)
__device__ __forceinline__ int pass_mo(int loc, int no, const int* occ0, const int* virt0, int g) {
    return loc < no ? occ0[g] + loc : virt0[g] + (loc - no);
}

template <typename T>
__global__ void k_ortho_eta(int w, const int* __restrict__ oblk, int n_oblk, const int* __restrict__ gnb_row,
                            const int* __restrict__ gnb_col, const int* __restrict__ group_nmol,
                            const int* __restrict__ group_not, const int* __restrict__ occ0,
                            const int* __restrict__ virt0, const int* __restrict__ blk_tp,
                            const T* __restrict__ sig, const double* __restrict__ dsc, DeviceScalars* sc,
                            const int* __restrict__ group_cl, double* __restrict__ cl_eta) {
    const int e = oblk[blockIdx.x];
    const int A = gnb_row[e], B = gnb_col[e];
    const int noA = 4 * group_nmol[A], noB = 4 * group_nmol[B];
    const int nA = w == 1 ? noA : 6 * group_nmol[A], nB = w == 1 ? noB : 6 * group_nmol[B];
    const bool same = A == B;
    double mx = 0.0;
    for (int p = threadIdx.x; p < nA * nB; p += blockDim.x) {
        const int i = p / nB, j = p % nB;
        if (same && j <= i) continue;
        int ia, ci, ib, cj;
        side_pos(i, noA, group_not[A], ia, ci);
        side_pos(j, noB, group_not[B], ib, cj);
        const double di = dsc[pass_mo(i, noA, occ0, virt0, A)], dj = dsc[pass_mo(j, noB, occ0, virt0, B)];
        mx = fmax(mx, fabs(sig_hat(sig, blk_tp, e, same, ia, ib, ci, cj, di, dj)));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(&sc->eta, mx);
        atomic_max_pos(&cl_eta[group_cl[A]], mx);
    }
}

template <typename T>
__global__ void k_ortho_lists(int w, double tol, const int* __restrict__ oblk, const int* __restrict__ gnb_row,
                              const int* __restrict__ gnb_col, const int* __restrict__ group_nmol,
                              const int* __restrict__ group_not, const int* __restrict__ occ0,
                              const int* __restrict__ virt0, const int* __restrict__ blk_tp,
                              const T* __restrict__ sig, const double* __restrict__ dsc, DeviceScalars* sc,
                              const int* __restrict__ group_cl, const double* __restrict__ cl_eta,
                              int* __restrict__ pr_n, int* __restrict__ pr_lvl, uint16_t* __restrict__ pr_ij,
                              T* __restrict__ pr_cs, int* __restrict__ pr_touch) {
    __shared__ unsigned char keep[48 * 48];
    __shared__ double s_sh[48 * 48];   // the normalised overlap of every kept pair
    __shared__ int cnt[kMaxSub + 1];
    const int e = oblk[blockIdx.x];
    const int A = gnb_row[e], B = gnb_col[e];
    const int noA = 4 * group_nmol[A], noB = 4 * group_nmol[B];
    const int nA = w == 1 ? noA : 6 * group_nmol[A], nB = w == 1 ? noB : 6 * group_nmol[B];
    const bool same = A == B;
    const int nsub = max(nA, nB);
    const double eta = cl_eta[group_cl[A]];   // threshold of the block's own cluster
    const bool active = !(eta < tol);
    const double cut = 1e-3 * eta;
    __shared__ int s_touch;
    if (threadIdx.x == 0) s_touch = 0;
    __syncthreads();
    int touch_t = 0;   // side tiles this thread's kept pairs touch: bits 0-2 side A, 3-5 side B
    for (int p = threadIdx.x; p < 48 * 48; p += blockDim.x) {
        const int i = p / 48, j = p % 48;
        unsigned char kp = 0;
        if (active && i < nA && j < nB && !(same && j <= i)) {
            int ia, ci, ib, cj;
            side_pos(i, noA, group_not[A], ia, ci);
            side_pos(j, noB, group_not[B], ib, cj);
            const double di = dsc[pass_mo(i, noA, occ0, virt0, A)], dj = dsc[pass_mo(j, noB, occ0, virt0, B)];
            const double sh = sig_hat(sig, blk_tp, e, same, ia, ib, ci, cj, di, dj);
            kp = fabs(sh) >= cut ? 1 : 0;
            if (kp) {
                touch_t |= (1 << ia) | (1 << (3 + ib));
                s_sh[p] = sh;
            }
        }
        keep[p] = kp;
    }
    if (touch_t) atomicOr(&s_touch, touch_t);
    __syncthreads();
    if ((int)threadIdx.x < nsub) {
        const int s = threadIdx.x;
        int c = 0;
        for (int i = 0; i < nA; ++i) {
            int j = ((s - i) % nsub + nsub) % nsub;
            if (j < nB && keep[i * 48 + j]) ++c;
        }
        cnt[s] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        int* lvl = pr_lvl + (size_t)e * (kMaxSub + 1);
        for (int s = 0; s < nsub; ++s) {
            lvl[s] = run;
            run += cnt[s];
        }
        for (int s = nsub; s <= kMaxSub; ++s) lvl[s] = run;
        pr_n[e] = run;
        if (run) atomicAdd(&sc->n_combo, (unsigned long long)run);
        pr_touch[e] = s_touch;
    }
    __syncthreads();
    if ((int)threadIdx.x < nsub) {
        const int s = threadIdx.x;
        int pos = pr_lvl[(size_t)e * (kMaxSub + 1) + s];
        for (int i = 0; i < nA; ++i) {
            int j = ((s - i) % nsub + nsub) % nsub;
            if (!(j < nB && keep[i * 48 + j])) continue;
            const double sh = s_sh[i * 48 + j];
            const size_t q = (size_t)e * kOrthoCap + pos;
            pr_ij[q] = (uint16_t)(i | (j << 8));
            pr_cs[2 * q] = (T)__dmul_rn(0.5, sh);
            pr_cs[2 * q + 1] = (T)0;
            ++pos;
        }
    }
}

// --------------------------------------------------------------------------
// Structural fill of a sweep (value-independent), then block-major apply.
//
// A unit is the set of tiles a block side touches: (group, occupied) and
// (group, virtual) for rotations and occupied passes, the whole group for
// passes over all MOs. A 2x2 update of an active block (one with pairs) can
// fill one side from the other, so before the sweep every row block is
// closed under "a block with pairs has both of its sides or neither"; all
// tiles of the units it holds are inserted as zero tiles. After that no
// update creates a tile: the sweep runs colour by colour, block-major, in
// place, and a final compaction drops the tiles left all-zero.
// --------------------------------------------------------------------------
struct SweepArgs {
    int mode;        // 0 rotations (A occupied | B virtual), 1 combinations
    int which;       // combinations: 0 all MOs, 1 occupied MOs
    int n_tiles, n_occ_tiles, n_groups, cap, n_blk, max_cl_groups, n_clusters;
    double trunc;
    float trunc_f;   // smallest float >= trunc: |x| < trunc <=> |x| < trunc_f for every float x
    const int* blk;          // blocks of the pass by colour
    const int* mol_cluster;  // closure: cluster of every row block
    const int* cl_g0;        // closure: first group, occupied tile and virtual tile of every cluster
    const int* cl_ot0;
    const int* cl_vt0;
    const int* clblk_ptr;    // closure: blocks of the pass by cluster
    const int* clblk;
    const int* unit_lab;     // closure: component label of every unit (2 per group), cluster-local
    int* lab_start;          // closure: per label, first entry of its members in lab_mem, and their count
    int* lab_cnt;
    int* lab_mem;            // closure: the units of every component, in increasing order
    const int* gnb_colour;   // closure: colour of every block ...
    int col_lo, col_hi;      // ... only blocks of colours [col_lo, col_hi) link units
    const int* gnb_row;
    const int* gnb_col;
    const int* group_nmol;
    const int* group_ot0;
    const int* group_not;
    const int* group_vt0;
    const int* group_nvt;
    const int* tile_group;
    const int* tile_kind;
    const int* tile_mo0;
    const int* tile_nmo;
    const int* pr_n;
    const int* pr_lvl;
    const int* pr_touch;     // tiles of each side a block's pairs touch: bits 0-2 side A, 3-5 side B
    const uint16_t* pr_ij;
    const void* pr_cs;
    const double* dsc;       // combinations: divide the pass's MOs by d_i first ...
    const double* cl_eta;    // ... in clusters whose eta is not below the pass's target
    double tol;              // (below it the pass has converged and changes nothing)
    unsigned long long* upd; // counter of 2x2 row updates
    const int* cci_ptr;
    const int* cci_row;
    const int* cci_slot;
    const int* in_nt;
    const int* in_tile;
    const void* in_val;
    int* out_nt;
    int* out_tile;
    void* out_val;
    unsigned char* out_nz;   // flags of out: 0 = the tile is all zero (written by the closure, kept by the sweep)
    unsigned char* col_nz;   // sweeps: the same flags in column-index order (entry p of cci_row / cci_slot)
    const int4* blk_info;    // FP32 sweeps: per block in colour order, (e, pairs, touch, rows), (pa, pb, rows of B, 0)
    const unsigned char* in_nz;   // closure: flags of the input (NULL: every listed tile may be nonzero)
    int normalise_pass;      // closure in mode 1: divide by d_i (the first closure of a pass)
    unsigned* err;
};


// truncation test |x| < threshold, decided exactly in the storage precision
__device__ __forceinline__ bool below(double x, const SweepArgs& a) { return fabs(x) < a.trunc; }
__device__ __forceinline__ bool below(float x, const SweepArgs& a) { return fabsf(x) < a.trunc_f; }
static_assert(sizeof(float) == 4, "");

// Connected components of a pass's units (the occupied or the virtual tiles
// of one group) under its active blocks, one CTA per cluster. The closure of a
// row is then the set of units whose component holds a unit the row has:
// "a block with pairs has both of its sides or neither", applied until nothing
// changes, is exactly that. Unit u of a cluster with ng groups: occupied
// tiles of local group u (u < ng), virtual tiles of local group u - ng.
// Hook-and-compress: roots are linked to the smaller root across every active
// block, then every label is replaced by its root, until no block links two
// roots. A label only ever points to a smaller unit of the same component.
__global__ void __launch_bounds__(1024) k_closure_labels(SweepArgs a, int* __restrict__ unit_lab) {
    extern __shared__ int slab[];   // 2 ng labels
    const int k = blockIdx.x;
    const int g0 = a.cl_g0[k], ng = a.cl_g0[k + 1] - g0, nu = 2 * ng;
    const int jb0 = a.clblk_ptr[k], jb1 = a.clblk_ptr[k + 1];
    const bool groups = a.mode == 1 && a.which == 0;   // occupied and virtual tiles of a group move together
    for (int u = threadIdx.x; u < nu; u += blockDim.x) slab[u] = u;
    __syncthreads();
    auto find = [&](int u) {
        int v = slab[u];
        while (v != u) {
            u = v;
            v = slab[u];
        }
        return u;
    };
    // every round that links at least one pair of roots removes a root, so at
    // most nu rounds can change anything
    for (int it = 0; it <= nu; ++it) {
        int changed = 0;
        const int n_edges = (jb1 - jb0) + (groups ? ng : 0);
        for (int j = threadIdx.x; j < n_edges; j += blockDim.x) {
            int u, v;
            if (j < jb1 - jb0) {
                const int e = a.clblk[jb0 + j];
                if (a.pr_n[e] == 0) continue;
                const int col = a.gnb_colour[e];
                if (col < a.col_lo || col >= a.col_hi) continue;
                u = a.gnb_row[e] - g0;
                v = a.mode == 0 ? ng + (a.gnb_col[e] - g0) : a.gnb_col[e] - g0;
            } else {
                u = j - (jb1 - jb0);
                v = ng + u;
            }
            const int ru = find(u), rv = find(v);
            if (ru != rv) {
                atomicMin(&slab[max(ru, rv)], min(ru, rv));
                changed = 1;
            }
        }
        const int any = __syncthreads_or(changed);
        for (int u = threadIdx.x; u < nu; u += blockDim.x) slab[u] = find(u);
        __syncthreads();
        if (!any) break;
    }
    for (int u = threadIdx.x; u < nu; u += blockDim.x) unit_lab[2 * g0 + u] = slab[u];
    // The members of every component in increasing unit order (CSR by label):
    // counts, an exclusive scan, then one warp places the units in order, the
    // lanes of a group of 32 with equal labels taking consecutive entries.
    int* cnt = slab + nu;
    for (int u = threadIdx.x; u < nu; u += blockDim.x) cnt[u] = 0;
    __syncthreads();
    for (int u = threadIdx.x; u < nu; u += blockDim.x) atomicAdd(&cnt[slab[u]], 1);
    __syncthreads();
    __shared__ int part[1024];
    const int per = (nu + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(nu, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int i = lo; i < hi; ++i) {
        const int c = cnt[i];
        a.lab_start[2 * g0 + i] = run;
        a.lab_cnt[2 * g0 + i] = c;
        cnt[i] = run;   // from here on: the next free entry of label i
        run += c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int base = 0; base < nu; base += 32) {
            const int u = base + lane;
            const unsigned act = __ballot_sync(0xffffffffu, u < nu);
            if (u < nu) {
                const int l = slab[u];
                const unsigned peers = __match_any_sync(act, l);
                a.lab_mem[2 * g0 + cnt[l] + __popc(peers & ((1u << lane) - 1u))] = u;
                __syncwarp(act);   // every peer has read cnt[l] before its first lane moves it
                if (lane == __ffs(peers) - 1) cnt[l] += __popc(peers);
            }
            __syncwarp();
        }
    }
}

// Components with more members than this are marked by a whole warp.
constexpr int kSmallComp = 8;
constexpr int kBigMax = 64;   // large components listed per row (more: marked by their claimant)
template <typename T>
__global__ void __launch_bounds__(256) k_closure(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    if (*a.err & (kErrCapacity | kErrSortSize)) return;   // an earlier kernel of the step overflowed
    // everything a row block touches belongs to its own cluster: units and
    // labels are indexed inside the cluster's ranges
    const int r = blockIdx.x;
    const int k = a.mol_cluster[r];
    const int g0 = a.cl_g0[k], ng = a.cl_g0[k + 1] - g0, nu = 2 * ng;
    const int uw = (2 * a.max_cl_groups + 31) >> 5;   // words of a bitset over a cluster's units
    const int nw = (nu + 31) >> 5;
    unsigned* present = (unsigned*)smraw;      // by label: components holding a nonzero tile of the row
    unsigned* onu = present + uw;              // by unit: units of the new row
    int* wpos = (int*)(onu + uw);              // per word of onu: its tile count, then its first slot
    int* oldt = wpos + uw;                     // the row's tile ids (sorted)
    short* oslot = (short*)(oldt + a.cap);     // per new slot: its slot in the row, or -1
    __shared__ int s_big[kBigMax];
    __shared__ int s_nbig;
    __shared__ int part[256];
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int* lab = a.unit_lab + 2 * g0;
    const int* lstart = a.lab_start + 2 * g0;
    const int* lcnt = a.lab_cnt + 2 * g0;
    const int* lmem = a.lab_mem + 2 * g0;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) present[i] = onu[i] = 0u;
    if (threadIdx.x == 0) s_nbig = 0;
    const int n0 = a.in_nt[r];
    for (int s = threadIdx.x; s < n0; s += blockDim.x) oldt[s] = a.in_tile[(size_t)r * a.cap + s];
    __syncthreads();
    auto mark = [&](int l, int j0, int dj) {
        const int m0 = lstart[l], mn = lcnt[l];
        for (int j = j0; j < mn; j += dj) {
            const int m = lmem[m0 + j];
            atomicOr(&onu[m >> 5], 1u << (m & 31));
        }
    };
    // The row keeps every unit of every component that holds one of its
    // nonzero tiles: a tile flagged all-zero keeps nothing and creates no fill.
    // The first thread to claim a component marks its members (a large one is
    // listed for a warp instead).
    for (int s = threadIdx.x; s < n0; s += blockDim.x) {
        if (a.in_nz && !a.in_nz[(size_t)r * a.cap + s]) continue;
        const int t = oldt[s];
        const int g = a.tile_group[t] - g0;
        const int u = ((a.mode == 1 && a.which == 0) || a.tile_kind[t] == 0) ? g : ng + g;
        const int l = lab[u];
        const unsigned bit = 1u << (l & 31);
        if (atomicOr(&present[l >> 5], bit) & bit) continue;
        if (lcnt[l] > kSmallComp) {
            const int i = atomicAdd(&s_nbig, 1);
            if (i < kBigMax) {
                s_big[i] = l;
                continue;
            }
        }
        mark(l, 0, 1);
    }
    __syncthreads();
    const int nbig = min(s_nbig, kBigMax);
    for (int b = warp; b < nbig; b += nwarps) mark(s_big[b], lane, 32);
    __syncthreads();
    // tiles per word of the new unit set, then their first slots (units in
    // order: occupied units by group, then virtual ones, i.e. tile ids ascending)
    auto ntiles = [&](int u) { return u < ng ? a.group_not[g0 + u] : a.group_nvt[g0 + u - ng]; };
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        unsigned b = onu[w];
        int c = 0;
        while (b) {
            c += ntiles(32 * w + __ffs(b) - 1);
            b &= b - 1;
        }
        wpos[w] = c;
    }
    __syncthreads();
    const int per = (nw + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(nw, w0 + per);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += wpos[w];
    part[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
        s_total = run;
    }
    __syncthreads();
    const int n1 = s_total;
    if (n1 > a.cap) {
        if (threadIdx.x == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    {
        int run = part[threadIdx.x];
        for (int w = w0; w < w1; ++w) {
            const int c = wpos[w];
            wpos[w] = run;
            run += c;
        }
    }
    __syncthreads();
    // the new row: tile ids, the slot each had in the row (binary search of the
    // sorted old list), flags: tiles that were in the row survived the last
    // compaction (or come from the guess or a restart) and may be nonzero;
    // inserted tiles are zero
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        unsigned b = onu[w];
        int pos = wpos[w];
        while (b) {
            const int u = 32 * w + __ffs(b) - 1;
            b &= b - 1;
            const int g = u < ng ? u : u - ng;
            const int t0 = u < ng ? a.group_ot0[g0 + g] : a.group_vt0[g0 + g];
            const int nt = ntiles(u);
            for (int i = 0; i < nt; ++i, ++pos) {
                const int t = t0 + i;
                int lo = 0, hi = n0;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (oldt[mid] < t) lo = mid + 1;
                    else hi = mid;
                }
                const int os = lo < n0 && oldt[lo] == t ? lo : -1;
                a.out_tile[(size_t)r * a.cap + pos] = t;
                oslot[pos] = (short)os;
                a.out_nz[(size_t)r * a.cap + pos] = os < 0 ? 0 : (a.in_nz ? a.in_nz[(size_t)r * a.cap + os] : 1);
            }
        }
    }
    if (threadIdx.x == 0) a.out_nt[r] = n1;
    __syncthreads();
    // values, 16 bytes at a time
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int kVec = 16 / (int)sizeof(T);
    constexpr int kPer = kTileVals / kVec;   // 16-byte pieces per tile
    const V* inv = (const V*)a.in_val + (size_t)r * a.cap * kPer;
    V* outv = (V*)a.out_val + (size_t)r * a.cap * kPer;
    const bool normalise = a.mode == 1 && a.normalise_pass && !(a.cl_eta[k] < a.tol);
    for (int idx = threadIdx.x; idx < n1 * kPer; idx += blockDim.x) {
        const int s = idx / kPer, piece = idx - s * kPer;
        const int os = oslot[s];
        V v;
        if (os >= 0) {
            v = inv[(size_t)os * kPer + piece];
            const int t = a.out_tile[(size_t)r * a.cap + s];
            if (normalise && (a.which == 0 || a.tile_kind[t] == 0)) {
                T* e = (T*)&v;
                const int nmo = a.tile_nmo[t], mo0 = a.tile_mo0[t];
#pragma unroll
                for (int q = 0; q < kVec; ++q) {
                    const int col = (piece * kVec + q) & 15;
                    if (col < nmo) e[q] = e[q] / (T)a.dsc[mo0 + col];
                }
            }
        } else {
            T* e = (T*)&v;
#pragma unroll
            for (int q = 0; q < kVec; ++q) e[q] = (T)0;
        }
        outv[(size_t)s * kPer + piece] = v;
    }
}


// The tile flags of the sweep's input in column-index order: entry p of tile
// t's list (row cci_row[p], slot cci_slot[p]) gets the flag of that tile in
// that row. The sweep kernels then test a block's rows for work with
// contiguous reads of its tiles' column lists, with no dependence on the slot
// loads, and raise both copies of a flag together. One CTA per tile.
__global__ void __launch_bounds__(256) k_flags_by_column(int cap, const int* __restrict__ cci_ptr,
                                                         const int* __restrict__ cci_row,
                                                         const int* __restrict__ cci_slot,
                                                         const unsigned char* __restrict__ nz,
                                                         unsigned char* __restrict__ col_nz) {
    const int t = blockIdx.x;
    const int lo = cci_ptr[t], hi = cci_ptr[t + 1];
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) col_nz[p] = nz[(size_t)cci_row[p] * cap + cci_slot[p]];
}

// What a CTA of k_apply_full needs to start on block q of the pass (colour
// order), gathered once per sweep so that it costs one load instead of a
// chain of dependent ones: the block, its pair count and touched tiles, and
// the column lists of the first tile of each side.
template <int MODE>
__global__ void k_block_info(SweepArgs a, int n, int4* __restrict__ info) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int e = a.blk[q];
    const int A = a.gnb_row[e], B = a.gnb_col[e];
    const int ta0 = a.group_ot0[A], tb0 = MODE == 0 ? a.group_vt0[B] : a.group_ot0[B];
    const int pa = a.cci_ptr[ta0], pb = a.cci_ptr[tb0];
    info[2 * q] = make_int4(e, a.pr_n[e], a.pr_touch[e], a.cci_ptr[ta0 + 1] - pa);
    info[2 * q + 1] = make_int4(pa, pb, a.cci_ptr[tb0 + 1] - pb, 0);
}

// side tiles of a block: up to 3 per side, as (first tile of a run, offset)
struct Side {
    int n;           // tiles on the side
    int run0;        // first tile of the occupied (or only) run
    int nrun0;       // tiles in that run
    int run1;        // first tile of the virtual run (all-MO passes) or -1
};

__device__ __forceinline__ Side side_of(const SweepArgs& a, int g, bool virt_only, bool with_virt) {
    Side s;
    if (virt_only) {
        s.run0 = a.group_vt0[g];
        s.nrun0 = a.group_nvt[g];
        s.run1 = -1;
        s.n = s.nrun0;
    } else {
        s.run0 = a.group_ot0[g];
        s.nrun0 = a.group_not[g];
        s.run1 = with_virt ? a.group_vt0[g] : -1;
        s.n = s.nrun0 + (with_virt ? a.group_nvt[g] : 0);
    }
    return s;
}

constexpr int kUnroll = 1;                 // pairs of one level in flight per thread (measured best)
constexpr int kSegUnroll = 4;              // panel segments in flight per thread

template <typename T> struct Vec;
template <> struct Vec<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <> struct Vec<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
};

// Rows per thread and row blocks per CTA: FP32 panels are processed two
// adjacent AO rows per thread with packed f32x2 arithmetic; FP64 one row.
template <typename T> struct ApplyShape;
template <> struct ApplyShape<float> {
    static constexpr int rows = 2, chunk = 64;
};
template <> struct ApplyShape<double> {
    static constexpr int rows = 1, chunk = 32;
};
template <typename T> __host__ __device__ constexpr int apply_nr() { return ApplyShape<T>::chunk * kAoPerMol; }
// even, bank-spread panel stride
template <typename T> __host__ __device__ constexpr int apply_nrp() { return apply_nr<T>() + 2; }
template <typename T> __host__ __device__ constexpr int apply_threads() { return apply_nr<T>() / ApplyShape<T>::rows; }

__device__ __forceinline__ float2 trunc2(float2 v, float t) {
    v.x = fabsf(v.x) < t ? 0.f : v.x;
    v.y = fabsf(v.y) < t ? 0.f : v.y;
    return v;
}

// One CTA = one active block of the colour x a chunk of row blocks. The
// block's side tiles of those rows are staged in shared memory as a
// [tile][column][row] panel; every thread owns one (FP64) or two adjacent
// (FP32) AO rows and applies the block's pairs to them in schedule order,
// level by level. Rows are independent, so no barrier is needed between
// levels; pairs of one level touch disjoint MOs, so kUnroll of them are
// loaded, updated and stored together.
template <typename T, int MODE, int NT, int PCAP>
__global__ void __launch_bounds__(apply_threads<T>()) k_apply_colour(SweepArgs a, int p0) {
    constexpr int CH = ApplyShape<T>::chunk, NRP = apply_nrp<T>();
    extern __shared__ __align__(16) unsigned char smraw[];
    T* panel = (T*)smraw;                                    // [NT tiles][16][NRP]
    T* pcs = panel + NT * 16 * NRP;                          // np * 2 coefficients
    unsigned* poff = (unsigned*)(pcs + 2 * PCAP);            // np packed panel offsets
    __shared__ int s_lvl[kMaxSub + 1];
    __shared__ int s_row[CH];
    __shared__ int s_slot[CH][NT];
    __shared__ int s_cp[NT];   // start of each panel tile's column list (-1: not held)
    // side A occupies panel tiles [0, kSideA), side B [kSideA, NT)
    constexpr int kSideA = MODE == 0 ? 2 : NT / 2;
    if (*a.err & (kErrCapacity | kErrSortSize)) return;
    const int e = a.blk[p0 + blockIdx.y];
    const int np = a.pr_n[e];
    if (np == 0) return;
    const int A = a.gnb_row[e], B = a.gnb_col[e];
    const bool with_virt = MODE == 1 && a.which == 0;
    const Side sa = side_of(a, A, false, with_virt);
    const Side sb = side_of(a, B, MODE == 0, with_virt);
    const int pa = a.cci_ptr[sa.run0], n_rows = a.cci_ptr[sa.run0 + 1] - pa;
    const int pb = a.cci_ptr[sb.run0];
    const int k0 = blockIdx.x * CH;
    if (k0 >= n_rows) return;
    if (a.cci_ptr[sb.run0 + 1] - pb != n_rows) {
        if (threadIdx.x == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    const int nk = min(CH, n_rows - k0);
    if (threadIdx.x == 0) atomicAdd(a.upd, (unsigned long long)np * (unsigned long long)(nk * 6));
    // a combination block inside one group: both sides are the same tiles, held once
    const bool same = MODE == 1 && A == B;
    const int pav = sa.run1 >= 0 ? a.cci_ptr[sa.run1] : 0;
    const int pbv = sb.run1 >= 0 ? a.cci_ptr[sb.run1] : 0;
    for (int t = threadIdx.x; t < nk; t += blockDim.x) {
        const int k = k0 + t;
        s_row[t] = a.cci_row[pa + k];
        const int so = a.cci_slot[pa + k];
        const int sv = sa.run1 >= 0 ? a.cci_slot[pav + k] : 0;
        const int bo = a.cci_slot[pb + k];
        const int bv = sb.run1 >= 0 ? a.cci_slot[pbv + k] : 0;
        for (int i = 0; i < NT / 2 + (NT & 1); ++i) {
            if (i < kSideA) s_slot[t][i] = i < sa.nrun0 ? so + i : (i < sa.n ? sv + (i - sa.nrun0) : -1);
            if (i < NT - kSideA)
                s_slot[t][kSideA + i] = same ? -1 : (i < sb.nrun0 ? bo + i : (i < sb.n ? bv + (i - sb.nrun0) : -1));
        }
    }
    if (threadIdx.x < NT) {
        const int p = threadIdx.x;
        int tile = -1;
        if (p < kSideA) {
            if (p < sa.nrun0) tile = sa.run0 + p;
            else if (p < sa.n) tile = sa.run1 + (p - sa.nrun0);
        } else if (!same) {
            const int i = p - kSideA;
            if (i < sb.nrun0) tile = sb.run0 + i;
            else if (i < sb.n) tile = sb.run1 + (i - sb.nrun0);
        }
        s_cp[p] = tile >= 0 ? a.cci_ptr[tile] : -1;
    }
    __syncthreads();
    // a chunk whose held tiles are all flagged zero in all its rows stays as it
    // is (the updates of zeros are zeros): nothing to load, update or store
    bool work = false;
    for (int t = threadIdx.x; t < nk; t += blockDim.x)
        for (int p = 0; p < NT; ++p) work |= s_cp[p] >= 0 && a.col_nz[s_cp[p] + k0 + t];
    if (!__syncthreads_or(work)) return;
    const int* lvl = a.pr_lvl + (size_t)e * (kMaxSub + 1);
    for (int i = threadIdx.x; i <= kMaxSub; i += blockDim.x) s_lvl[i] = lvl[i];
    const T* cs = (const T*)a.pr_cs + (size_t)e * kOrthoCap * 2;
    const uint16_t* ij = a.pr_ij + (size_t)e * kOrthoCap;
    const int noA = 4 * a.group_nmol[A], noB = 4 * a.group_nmol[B];
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const unsigned w = ij[q];
        const int il = w & 255, jl = w >> 8;
        int ta, ca, tb, cb;
        if (MODE == 0) {
            ta = il >> 4;
            ca = il & 15;
            tb = kSideA + (jl >> 4);
            cb = jl & 15;
        } else {
            side_pos(il, noA, sa.nrun0, ta, ca);
            side_pos(jl, noB, sb.nrun0, tb, cb);
            if (!same) tb += kSideA;
        }
        poff[q] = (unsigned)((ta * 16 + ca) * NRP) | ((unsigned)((tb * 16 + cb) * NRP) << 16);
        pcs[2 * q] = cs[2 * q];
        pcs[2 * q + 1] = cs[2 * q + 1];
    }
    __syncthreads();
    T* val = (T*)a.out_val;   // in place
    // panel load: one 16-value AO-row segment (rb, p, k) per item, vector loads,
    // kSegUnroll segments in flight per thread, transposed into the panel
    using V = typename Vec<T>::type;
    constexpr int kVPer = 16 / Vec<T>::n;   // vector loads per segment
    const int nseg = nk * 6 * NT;
    for (int s0 = threadIdx.x; s0 < nseg; s0 += blockDim.x * kSegUnroll) {
        V buf[kSegUnroll][kVPer];
#pragma unroll
        for (int u = 0; u < kSegUnroll; ++u) {
            const int sg = s0 + u * blockDim.x;
            if (sg < nseg) {
                const int rb = sg / (6 * NT), rem = sg - rb * (6 * NT), p = rem / 6, kr = rem - p * 6;
                const int sl = s_slot[rb][p];
                if (sl >= 0) {
                    const V* src = (const V*)(val + ((size_t)s_row[rb] * a.cap + sl) * kTileVals + kr * 16);
#pragma unroll
                    for (int v = 0; v < kVPer; ++v) buf[u][v] = src[v];
                } else {
#pragma unroll
                    for (int v = 0; v < kVPer; ++v) buf[u][v] = Vec<T>::zero();
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kSegUnroll; ++u) {
            const int sg = s0 + u * blockDim.x;
            if (sg < nseg) {
                const int rb = sg / (6 * NT), rem = sg - rb * (6 * NT), p = rem / 6, kr = rem - p * 6;
                const T* e2 = (const T*)buf[u];
                T* dst = panel + (p * 16) * NRP + rb * 6 + kr;
#pragma unroll
                for (int col = 0; col < 16; ++col) dst[col * NRP] = e2[col];
            }
        }
    }
    __syncthreads();
    constexpr int R = ApplyShape<T>::rows;
    const int row = threadIdx.x * R;
    // a warp whose rows hold only zeros in the block's tiles has nothing to update
    bool nzrow = false;
    if (row < nk * 6)
        for (int cidx = 0; cidx < NT * 16 && !nzrow; ++cidx)
#pragma unroll
            for (int r2 = 0; r2 < R; ++r2) nzrow |= panel[cidx * NRP + row + r2] != (T)0;
    const bool warp_busy = __any_sync(0xffffffffu, nzrow);
    if (row < nk * 6 && warp_busy) {
        T* pr = panel + row;
        for (int sub = 0; sub < kMaxSub; ++sub) {
            const int q1 = s_lvl[sub + 1];
            int q = s_lvl[sub];
            if (q == np) break;
            for (; q < q1; q += kUnroll) {
                if constexpr (R == 2) {
                    unsigned off[kUnroll];
                    float2 x[kUnroll], y[kUnroll];
                    float c0[kUnroll], c1[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        if (q + u < q1) {
                            off[u] = poff[q + u];
                            c0[u] = pcs[2 * (q + u)];
                            c1[u] = pcs[2 * (q + u) + 1];
                            x[u] = *(const float2*)(pr + (off[u] & 0xffffu));
                            y[u] = *(const float2*)(pr + (off[u] >> 16));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        if (q + u < q1) {
                            float2 xn, yn;
                            if (MODE == 0) {
                                const float2 cc = make_float2(c0[u], c0[u]);
                                xn = __ffma2_rn(cc, x[u], __fmul2_rn(make_float2(c1[u], c1[u]), y[u]));
                                yn = __ffma2_rn(cc, y[u], __fmul2_rn(make_float2(-c1[u], -c1[u]), x[u]));
                            } else {
                                const float2 nh = make_float2(-c0[u], -c0[u]);
                                xn = __ffma2_rn(nh, y[u], x[u]);
                                yn = __ffma2_rn(nh, x[u], y[u]);
                            }
                            *(float2*)(pr + (off[u] & 0xffffu)) = trunc2(xn, a.trunc_f);
                            *(float2*)(pr + (off[u] >> 16)) = trunc2(yn, a.trunc_f);
                        }
                    }
                } else {
                    unsigned off[kUnroll];
                    T x[kUnroll], y[kUnroll], c0[kUnroll], c1[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        if (q + u < q1) {
                            off[u] = poff[q + u];
                            c0[u] = pcs[2 * (q + u)];
                            c1[u] = pcs[2 * (q + u) + 1];
                            x[u] = pr[off[u] & 0xffffu];
                            y[u] = pr[off[u] >> 16];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        if (q + u < q1) {
                            T xn, yn;
                            if (MODE == 0) {
                                xn = c0[u] * x[u] + c1[u] * y[u];
                                yn = c0[u] * y[u] - c1[u] * x[u];
                            } else {
                                xn = x[u] - c0[u] * y[u];
                                yn = y[u] - c0[u] * x[u];
                            }
                            pr[off[u] & 0xffffu] = below(xn, a) ? (T)0 : xn;
                            pr[off[u] >> 16] = below(yn, a) ? (T)0 : yn;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
        const int rb = sg / (6 * NT), rem = sg - rb * (6 * NT), p = rem / 6, kr = rem - p * 6;
        const int sl = s_slot[rb][p];
        if (sl < 0) continue;
        V out[kVPer];
        T* e2 = (T*)out;
        const T* srcp = panel + (p * 16) * NRP + rb * 6 + kr;
        bool any = false;
#pragma unroll
        for (int col = 0; col < 16; ++col) {
            e2[col] = srcp[col * NRP];
            any |= e2[col] != (T)0;
        }
        if (any) {   // the tile may be nonzero now
            a.out_nz[(size_t)s_row[rb] * a.cap + sl] = 1;
            a.col_nz[s_cp[p] + k0 + rb] = 1;
        }
        V* dst = (V*)(val + ((size_t)s_row[rb] * a.cap + sl) * kTileVals + kr * 16);
#pragma unroll
        for (int v = 0; v < kVPer; ++v) dst[v] = out[v];
    }
}

// Blocks between full groups (8 molecules: 32 occupied and 16 virtual MOs per
// group) in FP32 storage: rotations (MODE 0, A occupied x B virtual) and
// occupied-pass combinations (MODE 1, A occupied x B occupied, A != B). The
// in-block colour of such a block is (i + j) mod 32. Same updates, order and
// truncation as k_apply_colour, laid out for fewer shared-memory round trips:
// each thread owns a pair of adjacent AO rows; the 32 A-side values of those rows
// stay in registers (the index i is static once the slot loop is unrolled),
// the NB B-side values sit in a thread-private shared-memory panel indexed by
// j = (level - i) mod 32. The block's pairs are expanded into a dense
// [level][i] coefficient table with a selection mask per level. The level loop
// needs no barrier: a thread reads back only the panel rows it wrote.
// Row pairs whose touched tiles are all flagged zero (per-tile flags written by
// the closure and raised by the sweep) are skipped: the updates would leave
// those zeros as they are. The others are collected over several row chunks so
// that the level loop runs in full warps.
constexpr int kFullDenseMin = 12;                 // pairs in a level from which MODE 1 runs it without branches
constexpr int kFullBatch = 8;                     // slots loaded ahead in a branch-free level (multiple of 4)
constexpr int kFusedBatch = 4;                    // slots loaded ahead when two levels share a pass (even)
constexpr int kFullMinCtas[2] = {6, 5};          // resident CTAs per SM the register budget is cut for
constexpr int kFullWaves[2] = {16, 4};            // resident-CTA multiples per launch (fewer: more row chunks per CTA to collect from)
constexpr int kFullCH = 32;                       // row blocks per CTA
constexpr int kFullNR = kFullCH * kAoPerMol;      // AO rows per CTA (panel stride, floats)
constexpr int kFullThreads = kFullNR / 2;         // one pair of adjacent AO rows per thread (two pairs measured slower)
template <int MODE> struct FullShape;
template <> struct FullShape<0> {   // rotations: B = one virtual tile, coefficients (c, c, s, s)
    static constexpr int nb = 16;
    using Coef = float4;
};
template <> struct FullShape<1> {   // combinations: B = two occupied tiles, (-c, truncation threshold)
    static constexpr int nb = 32;
    using Coef = float2;
};
template <int MODE> __host__ __device__ constexpr size_t full_apply_smem() {
    return (size_t)FullShape<MODE>::nb * kFullNR * 4 + (size_t)32 * 32 * sizeof(typename FullShape<MODE>::Coef);
}

// 1.0 where |v| >= t, 0.0 below (and for NaN): one compare that writes the
// factor itself
__device__ __forceinline__ float ge_abs_factor(float v, float t) {
    float k;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(k) : "f"(fabsf(v)), "f"(t));
    return k;
}

// x with the values below t in magnitude set to zero, as a product with 0/1
// factors: two compares on the ALU pipe and one packed multiply on the FMA
// pipe instead of two compares and two selects (a value set to zero may come
// out as -0, which every later test treats as zero)
__device__ __forceinline__ float2 trunc2_mul(float2 v, float t) {
    return __fmul2_rn(v, make_float2(ge_abs_factor(v.x, t), ge_abs_factor(v.y, t)));
}

__device__ __forceinline__ void load_pair_rows(const float* src, float4 (&r0)[4], float4 (&r1)[4]) {
    const float4* s = (const float4*)src;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        r0[v] = s[v];
        r1[v] = s[4 + v];   // next AO row: 16 floats on
    }
}

template <int MODE>
__global__ void __launch_bounds__(kFullThreads, kFullMinCtas[MODE]) k_apply_full(SweepArgs a, int p0) {
    constexpr int NB = FullShape<MODE>::nb;
    using Coef = typename FullShape<MODE>::Coef;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* panel = (float*)smraw;                           // [NB B columns][kFullNR rows]
    Coef* coef = (Coef*)(panel + NB * kFullNR);             // [32 levels][32 i]
    __shared__ unsigned s_mask[32];
    if (*a.err & (kErrCapacity | kErrSortSize)) return;
    const int4 i0 = a.blk_info[2 * (p0 + blockIdx.y)], i1 = a.blk_info[2 * (p0 + blockIdx.y) + 1];
    const int e = i0.x, np = i0.y, touch = i0.z, n_rows = i0.w;
    const int pa = i1.x, pb = i1.y;
    if (np == 0) return;
    // CTA x takes row chunks x, x + gridDim.x, ... of the block, so its
    // coefficient table serves several chunks
    const int k_first = blockIdx.x * kFullCH;
    if (k_first >= n_rows) return;
    if (i1.z != n_rows) {
        if (threadIdx.x == 0) atomicOr(a.err, kErrCapacity);
        return;
    }
    // rotations read only the slots that hold a pair (the mask's bits); the
    // dense levels of occupied passes read every slot, so those start at zero
    if constexpr (MODE == 1)
        for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) coef[i] = make_float2(0.f, 0.f);
    if (threadIdx.x < 32) s_mask[threadIdx.x] = 0u;
    __syncthreads();
    const float* cs = (const float*)a.pr_cs + (size_t)e * kOrthoCap * 2;
    const uint16_t* ij = a.pr_ij + (size_t)e * kOrthoCap;
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const unsigned w = ij[q];
        const int il = w & 255, jl = w >> 8, lv = (il + jl) & 31;
        const float c = cs[2 * q];
        if constexpr (MODE == 0) {
            const float sn = cs[2 * q + 1];
            coef[lv * 32 + il] = make_float4(c, c, sn, sn);
        } else {
            coef[lv * 32 + il] = make_float2(-c, a.trunc_f);   // a slot without a pair keeps (0, 0)
        }
        atomicOr(&s_mask[lv], 1u << il);
    }
    __syncthreads();
    // tiles no selected pair touches (touch bits clear) keep their values:
    // neither loaded nor stored
    float* val = (float*)a.out_val;   // in place
    // The side tiles of a unit are consecutive tile ids with equal column
    // lists, so side tile t's list starts t * n_rows after the first one's.
    // Each row chunk first tells, per row pair, whether it has work: a row pair
    // whose touched tiles are all flagged zero stays zero under the block's
    // updates (x - c y and c x + s y of zeros, truncation keeps zeros), and so
    // does a flagged row pair of zeros that runs through them. The row pairs
    // with work are appended to a shared list; once it holds a CTA's worth,
    // every thread takes one, loads both sides and runs the updates, so that the
    // level loop runs in full warps. The rest runs at the end. The flags are
    // read in column-index order (contiguous for consecutive rows of the
    // block), together with the rows and slots the run needs.
    __shared__ int s_list[2 * kFullThreads];   // row pairs with work, not yet run
    __shared__ int s_lrow[2 * kFullThreads];   // their row block and the slots of both sides there
    __shared__ int s_lsa[2 * kFullThreads];
    __shared__ int s_lsb[2 * kFullThreads];
    __shared__ int s_wcnt[kFullThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = threadIdx.x / 3;   // own row block (of the chunk)
    // the updates of one row pair with work: entry = (row block in the block's
    // row list) * 3 + pair
    auto run = [&](const int ent, const int row, const int slA, const int slB) {
        const int kr = ent / 3, k2s = 2 * (ent - 3 * kr);
        const size_t baseA = ((size_t)row * a.cap + slA) * kTileVals + k2s * kTileW;
        const size_t baseB = ((size_t)row * a.cap + slB) * kTileVals + k2s * kTileW;
        // the B side goes to the thread's own panel rows (consecutive threads,
        // consecutive 8-byte words: no bank conflicts in the level loop)
        float* ps = panel + 2 * threadIdx.x;
#pragma unroll
        for (int t = 0; t < NB / 16; ++t) {
            float4 v0[4], v1[4];
            if (touch >> (3 + t) & 1) {
                load_pair_rows(val + baseB + (size_t)t * kTileVals, v0, v1);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) v0[v] = v1[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                *(float2*)(ps + (t * 16 + 4 * v + 0) * kFullNR) = make_float2(v0[v].x, v1[v].x);
                *(float2*)(ps + (t * 16 + 4 * v + 1) * kFullNR) = make_float2(v0[v].y, v1[v].y);
                *(float2*)(ps + (t * 16 + 4 * v + 2) * kFullNR) = make_float2(v0[v].z, v1[v].z);
                *(float2*)(ps + (t * 16 + 4 * v + 3) * kFullNR) = make_float2(v0[v].w, v1[v].w);
            }
        }
        float2 x[32];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            float4 u0[4], u1[4];
            if (touch >> t & 1) {
                load_pair_rows(val + baseA + (size_t)t * kTileVals, u0, u1);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) u0[v] = u1[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                x[t * 16 + 4 * v + 0] = make_float2(u0[v].x, u1[v].x);
                x[t * 16 + 4 * v + 1] = make_float2(u0[v].y, u1[v].y);
                x[t * 16 + 4 * v + 2] = make_float2(u0[v].z, u1[v].z);
                x[t * 16 + 4 * v + 3] = make_float2(u0[v].w, u1[v].w);
            }
        }
        const float tf = a.trunc_f;
        for (int lv = 0; lv < 32; ++lv) {
            const unsigned m = s_mask[lv];
            if (m == 0u) continue;
            const Coef* cl = coef + lv * 32;
            if constexpr (MODE == 1) {
                if (__popc(m) >= kFullDenseMin) {
                    // Most slots of the level hold a pair: all 32 run without a
                    // branch; a slot without a pair (c = 0, threshold 0) leaves
                    // both of its values as they are. Each slot reads (c, t) from
                    // the table, two slots per 16-byte load.
                    if (lv + 1 < 32 && __popc(s_mask[lv + 1]) >= kFullDenseMin) {
                        // Two dense levels in one pass over the slots. Slot i of
                        // level lv+1 pairs x_i with y_(lv+1-i), the value slot i-1
                        // has just updated at level lv: it stays in a register for
                        // its second update and is stored once. Slot 0's level-lv+1
                        // partner, y_(lv+1), is last updated at level lv by slot 31,
                        // so that update comes after the pass. Every value sees its
                        // updates in level order, as in the one-level pass.
                        const float4* ca4 = (const float4*)cl;
                        const float4* cb4 = (const float4*)(cl + 32);
                        float2 yprev = make_float2(0.f, 0.f);
#pragma unroll
                        for (int i0 = 0; i0 < 32; i0 += kFusedBatch) {
                            float2 yv[kFusedBatch];
                            float4 ca[kFusedBatch / 2], cb[kFusedBatch / 2];
#pragma unroll
                            for (int u = 0; u < kFusedBatch / 2; ++u) {
                                ca[u] = ca4[i0 / 2 + u];
                                cb[u] = cb4[i0 / 2 + u];
                            }
#pragma unroll
                            for (int u = 0; u < kFusedBatch; ++u)
                                yv[u] = *(const float2*)(ps + ((lv - i0 - u) & 31) * kFullNR);
#pragma unroll
                            for (int u = 0; u < kFusedBatch; ++u) {
                                const int i = i0 + u;
                                const float c0 = (u & 1) ? ca[u / 2].z : ca[u / 2].x;
                                const float t0 = (u & 1) ? ca[u / 2].w : ca[u / 2].y;
                                const float2 cc0 = make_float2(c0, c0);
                                const float2 xn = __ffma2_rn(cc0, yv[u], x[i]);
                                const float2 yn = __ffma2_rn(cc0, x[i], yv[u]);
                                x[i] = trunc2_mul(xn, t0);
                                const float2 ynew = trunc2_mul(yn, t0);
                                if (i > 0) {
                                    const float c1 = (u & 1) ? cb[u / 2].z : cb[u / 2].x;
                                    const float t1 = (u & 1) ? cb[u / 2].w : cb[u / 2].y;
                                    const float2 cc1 = make_float2(c1, c1);
                                    const float2 xn1 = __ffma2_rn(cc1, yprev, x[i]);
                                    const float2 yn1 = __ffma2_rn(cc1, x[i], yprev);
                                    x[i] = trunc2_mul(xn1, t1);
                                    *(float2*)(ps + ((lv + 1 - i) & 31) * kFullNR) = trunc2_mul(yn1, t1);
                                }
                                yprev = ynew;
                            }
                        }
                        {   // slot 0 of level lv+1 with y_(lv+1)
                            const float2 ct = cl[32];
                            const float2 cc1 = make_float2(ct.x, ct.x);
                            const float2 xn1 = __ffma2_rn(cc1, yprev, x[0]);
                            const float2 yn1 = __ffma2_rn(cc1, x[0], yprev);
                            x[0] = trunc2_mul(xn1, ct.y);
                            *(float2*)(ps + ((lv + 1) & 31) * kFullNR) = trunc2_mul(yn1, ct.y);
                        }
                        ++lv;
                        continue;
                    }
                    const float4* cl4 = (const float4*)cl;
#pragma unroll
                    for (int i0 = 0; i0 < 32; i0 += kFullBatch) {
                        float2 yv[kFullBatch];
                        float4 cv[kFullBatch / 2];
#pragma unroll
                        for (int u = 0; u < kFullBatch / 2; ++u) cv[u] = cl4[i0 / 2 + u];
#pragma unroll
                        for (int u = 0; u < kFullBatch; ++u)
                            yv[u] = *(const float2*)(ps + ((lv - i0 - u) & 31) * kFullNR);
#pragma unroll
                        for (int u = 0; u < kFullBatch; ++u) {
                            const int i = i0 + u;
                            const float c = (u & 1) ? cv[u / 2].z : cv[u / 2].x;
                            const float t = (u & 1) ? cv[u / 2].w : cv[u / 2].y;
                            const float2 cc = make_float2(c, c);
                            const float2 xn = __ffma2_rn(cc, yv[u], x[i]);
                            const float2 yn = __ffma2_rn(cc, x[i], yv[u]);
                            x[i] = trunc2_mul(xn, t);
                            *(float2*)(ps + ((lv - i) & 31) * kFullNR) = trunc2_mul(yn, t);
                        }
                    }
                    continue;
                }
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (m & (1u << i)) {
                    float2* py = (float2*)(ps + ((lv - i) & 31) * kFullNR);
                    const Coef c4 = cl[i];
                    const float2 y = *py;
                    float2 xn, yn;
                    if constexpr (MODE == 0) {
                        const float2 cc = make_float2(c4.x, c4.y);
                        xn = __ffma2_rn(cc, x[i], __fmul2_rn(make_float2(c4.z, c4.w), y));
                        yn = __ffma2_rn(cc, y, __fmul2_rn(make_float2(-c4.z, -c4.w), x[i]));
                    } else {
                        const float2 cc = make_float2(c4.x, c4.x);
                        xn = __ffma2_rn(cc, y, x[i]);
                        yn = __ffma2_rn(cc, x[i], y);
                    }
                    x[i] = trunc2(xn, tf);
                    *py = trunc2(yn, tf);
                }
            }
        }
        // store, and mark the tiles that hold a nonzero value now (a flag is
        // never cleared during the sweep: 1 only means "may be nonzero")
        unsigned char* f = a.out_nz + (size_t)row * a.cap;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (!(touch >> t & 1)) continue;
            float4* d0 = (float4*)(val + baseA + (size_t)t * kTileVals);
            bool any = false;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float2 a0 = x[t * 16 + 4 * v], a1 = x[t * 16 + 4 * v + 1];
                const float2 a2 = x[t * 16 + 4 * v + 2], a3 = x[t * 16 + 4 * v + 3];
                d0[v] = make_float4(a0.x, a1.x, a2.x, a3.x);
                d0[4 + v] = make_float4(a0.y, a1.y, a2.y, a3.y);
                any |= a0.x != 0.f || a0.y != 0.f || a1.x != 0.f || a1.y != 0.f || a2.x != 0.f ||
                       a2.y != 0.f || a3.x != 0.f || a3.y != 0.f;
            }
            if (any) {
                f[slA + t] = 1;
                a.col_nz[pa + t * n_rows + kr] = 1;
            }
        }
#pragma unroll
        for (int t = 0; t < NB / 16; ++t) {
            if (!(touch >> (3 + t) & 1)) continue;
            float4* d1 = (float4*)(val + baseB + (size_t)t * kTileVals);
            bool any = false;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float2 b0 = *(const float2*)(ps + (t * 16 + 4 * v + 0) * kFullNR);
                const float2 b1 = *(const float2*)(ps + (t * 16 + 4 * v + 1) * kFullNR);
                const float2 b2 = *(const float2*)(ps + (t * 16 + 4 * v + 2) * kFullNR);
                const float2 b3 = *(const float2*)(ps + (t * 16 + 4 * v + 3) * kFullNR);
                d1[v] = make_float4(b0.x, b1.x, b2.x, b3.x);
                d1[4 + v] = make_float4(b0.y, b1.y, b2.y, b3.y);
                any |= b0.x != 0.f || b0.y != 0.f || b1.x != 0.f || b1.y != 0.f || b2.x != 0.f ||
                       b2.y != 0.f || b3.x != 0.f || b3.y != 0.f;
            }
            if (any) {
                f[slB + t] = 1;
                a.col_nz[pb + t * n_rows + kr] = 1;
            }
        }
    };
    int n_acc = 0;   // entries in s_list (the same in every thread)
    int k0 = k_first;
    // one call site of the update code (it is large): collect row pairs until
    // a CTA's worth is listed or the block's rows run out, then run them
    for (;;) {
        while (n_acc < kFullThreads && k0 < n_rows) {
            const int nk = min(kFullCH, n_rows - k0);
            // the counter holds the 2x2 row updates the algorithm defines, rows proven
            // unchanged and skipped included
            if (threadIdx.x == 0) atomicAdd(a.upd, (unsigned long long)np * (unsigned long long)(nk * 6));
            bool work = false;
            int row = 0, slA = 0, slB = 0;
            if (rb < nk) {
                const int k = k0 + rb;
                row = a.cci_row[pa + k];
                slA = a.cci_slot[pa + k];
                slB = a.cci_slot[pb + k];
#pragma unroll
                for (int t = 0; t < 2; ++t) work |= (touch >> t & 1) && a.col_nz[pa + t * n_rows + k];
#pragma unroll
                for (int t = 0; t < NB / 16; ++t) work |= (touch >> (3 + t) & 1) && a.col_nz[pb + t * n_rows + k];
            }
            // pack the row pairs with work to the first threads
            const unsigned bal = __ballot_sync(0xffffffffu, work);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = 0, n_work = 0;
#pragma unroll
            for (int w = 0; w < kFullThreads / 32; ++w) {
                before += w < warp ? s_wcnt[w] : 0;
                n_work += s_wcnt[w];
            }
            if (work) {
                const int i = n_acc + before + __popc(bal & ((1u << lane) - 1u));
                s_list[i] = 3 * k0 + threadIdx.x;
                s_lrow[i] = row;
                s_lsa[i] = slA;
                s_lsb[i] = slB;
            }
            n_acc += n_work;
            k0 += gridDim.x * kFullCH;
            __syncthreads();
        }
        if (n_acc == 0) break;
        const int take = min(n_acc, kFullThreads);
        const bool mine = (int)threadIdx.x < take;
        int ent = 0, erow = 0, esa = 0, esb = 0;
        if (mine) {
            ent = s_list[threadIdx.x];
            erow = s_lrow[threadIdx.x];
            esa = s_lsa[threadIdx.x];
            esb = s_lsb[threadIdx.x];
        }
        __syncthreads();   // entries read: move the rest (fewer than a CTA's worth) to the front
        for (int i = threadIdx.x; i < n_acc - take; i += blockDim.x) {
            s_list[i] = s_list[take + i];
            s_lrow[i] = s_lrow[take + i];
            s_lsa[i] = s_lsa[take + i];
            s_lsb[i] = s_lsb[take + i];
        }
        n_acc -= take;
        if (mine) run(ent, erow, esa, esb);
        __syncthreads();   // the list is rewritten by the next chunk
    }
}

// drop tiles whose 6x16 values are all zero; in -> out
// (skipped entirely when an earlier kernel of the pass set the error word:
// `out` is then the pass's untouched input and stays as it was).
// One CTA per row block: a warp per tile marks the nonzero tiles in a shared
// bitmask, one thread turns the mask into word offsets, and the warps copy the
// nonzero tiles to their compacted slots (order kept); three barriers per row.
constexpr int kCompactMaxWords = 1024;   // 32768 slots (the 16-bit slot limit)
template <typename T>
__global__ void __launch_bounds__(256) k_compact(int cap, const int* __restrict__ in_nt,
                                                 const int* __restrict__ in_tile, const T* __restrict__ in_val,
                                                 int* __restrict__ out_nt, int* __restrict__ out_tile,
                                                 T* __restrict__ out_val, const unsigned* __restrict__ err) {
    __shared__ unsigned s_bits[kCompactMaxWords];
    __shared__ int s_pre[kCompactMaxWords];
    if (*err & (kErrCapacity | kErrSortSize)) return;
    const int r = blockIdx.x;
    const int n = in_nt[r];
    const int nw = (n + 31) >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int kPer = kTileVals * (int)sizeof(T) / 16;   // 16-byte pieces per tile (24 or 48)
    for (int i = threadIdx.x; i < nw; i += blockDim.x) s_bits[i] = 0u;
    __syncthreads();
    for (int s = warp; s < n; s += nwarps) {
        const VT* v = (const VT*)(in_val + ((size_t)r * cap + s) * kTileVals);
        bool nz = false;
        for (int i = lane; i < kPer; i += 32) {
            const VT x = v[i];
            if constexpr (sizeof(T) == 4)
                nz |= x.x != 0.f || x.y != 0.f || x.z != 0.f || x.w != 0.f;
            else
                nz |= x.x != 0.0 || x.y != 0.0;
        }
        if (__any_sync(0xffffffffu, nz) && lane == 0) atomicOr(&s_bits[s >> 5], 1u << (s & 31));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < nw; ++w) {
            s_pre[w] = run;
            run += __popc(s_bits[w]);
        }
        out_nt[r] = run;
    }
    __syncthreads();
    for (int s = warp; s < n; s += nwarps) {
        const unsigned w = s_bits[s >> 5];
        if (!(w >> (s & 31) & 1u)) continue;
        const int pos = s_pre[s >> 5] + __popc(w & ((1u << (s & 31)) - 1u));
        const VT* v = (const VT*)(in_val + ((size_t)r * cap + s) * kTileVals);
        VT* o = (VT*)(out_val + ((size_t)r * cap + pos) * kTileVals);
        for (int i = lane; i < kPer; i += 32) o[i] = v[i];
        if (lane == 0) out_tile[(size_t)r * cap + pos] = in_tile[(size_t)r * cap + s];
    }
}

}  // namespace

size_t closure_smem_bytes(const Ctx* c) {
    const size_t uw = (size_t)(2 * c->max_cl_groups + 31) / 32;
    return 3 * uw * 4 + (size_t)c->cap * 4 + (size_t)((c->cap + 1) & ~1) * 2 + 16;
}

size_t closure_labels_smem_bytes(const Ctx* c) { return (size_t)4 * c->max_cl_groups * 4; }

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
template <typename T>
static cudaError_t select_rot_t(Ctx* c) {
    const double tau = c->prm.eps;
    ClSel* cl = (ClSel*)c->d_cl_sel;
    // per-cluster state: counts and prefixes zero, kmax = rot_cap_factor * N_occ(cluster)
    cudaError_t e = cudaMemcpyAsync(c->d_cl_sel, c->d_cl_sel_init, c->h_cl_sel_init.size() * 8,
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
    k_rot_stats<T><<<c->n_gnb, 256, 0, c->stream>>>(c->n_gnb, c->d_gnb_row, c->d_gnb_col, c->d_group_nmol,
                                                    c->d_group_nvt, c->d_group_cl, c->d_rot_blk_tp0, (const T*)c->d_F,
                                                    tau, c->d_sc, cl);
    const int hb = std::min(c->n_gnb, 1024);
    // the keys are the bit patterns of |F| as doubles; a float widened to double
    // has its 29 lowest mantissa bits zero, so for FP32 storage the radix passes
    // below bit 24 would only ever pick bin 0 and are left out
    const int last = std::is_same<T, float>::value ? 24 : 0;
    for (int shift = 56; shift >= last; shift -= 8) {
        k_rot_hist<T><<<hb, 256, 0, c->stream>>>(shift, c->n_gnb, c->d_gnb_row, c->d_gnb_col, c->d_group_nmol,
                                                 c->d_group_nvt, c->d_group_cl, c->d_rot_blk_tp0, (const T*)c->d_F,
                                                 tau, cl, c->d_cl_hist);
        k_rot_pick<<<(c->n_clusters + 127) / 128, 128, 0, c->stream>>>(shift, last, c->n_clusters, cl, c->d_cl_hist);
    }
    k_rot_lists<T><<<c->n_gnb, 128, 0, c->stream>>>(
        c->n_gnb, c->d_gnb_row, c->d_gnb_col, c->d_group_nmol, c->d_group_nvt, c->d_group_occ0_mo,
        c->d_group_virt0_mo, c->d_group_cl, c->d_rot_blk_tp0, (const T*)c->d_F, c->d_Fd, tau, c->d_sc, cl, c->d_pr_n,
        c->d_pr_lvl, c->d_pr_ij, (T*)c->d_pr_cs, c->d_pr_touch);
    return cudaGetLastError();
}

cudaError_t launch_select_rot(Ctx* c) {
    c->n_launch += c->prec == SSCF_FP64 ? 2 + 2 * 8 : 2 + 2 * 5;   // stats, lists, radix passes (hist + pick)
    return c->prec == SSCF_FP64 ? select_rot_t<double>(c) : select_rot_t<float>(c);
}

template <typename T>
static cudaError_t ortho_prepare_t(Ctx* c, int w, double tol) {
    const int t_hi = w == 1 ? c->n_occ_tiles : c->n_tiles;
    k_ortho_scale<T><<<(t_hi * 16 + 255) / 256, 256, 0, c->stream>>>(
        w, 0, t_hi, c->d_tile_group, c->d_tile_kind, c->d_tile_nmo, c->d_tile_mo0, c->d_group_ot0, c->d_group_not,
        c->d_group_vt0, c->d_self_blk, c->d_ort_blk_tp[w], (const T*)c->d_sig, c->d_scale, &c->d_sc->err);
    const int nob = (int)c->h_ocolour_blk.size();
    cudaError_t e = cudaMemsetAsync(c->d_cl_eta, 0, (size_t)c->n_clusters * 8, c->stream);
    if (e != cudaSuccess) return e;
    k_ortho_eta<T><<<nob, 256, 0, c->stream>>>(w, c->d_ocolour_blk, nob, c->d_gnb_row, c->d_gnb_col,
                                              c->d_group_nmol, c->d_group_not, c->d_group_occ0_mo,
                                              c->d_group_virt0_mo, c->d_ort_blk_tp[w], (const T*)c->d_sig,
                                              c->d_scale, c->d_sc, c->d_group_cl, c->d_cl_eta);
    k_ortho_lists<T><<<nob, 128, 0, c->stream>>>(w, tol, c->d_ocolour_blk, c->d_gnb_row, c->d_gnb_col,
                                                c->d_group_nmol, c->d_group_not, c->d_group_occ0_mo,
                                                c->d_group_virt0_mo, c->d_ort_blk_tp[w], (const T*)c->d_sig,
                                                c->d_scale, c->d_sc, c->d_group_cl, c->d_cl_eta, c->d_pr_n,
                                                c->d_pr_lvl, c->d_pr_ij,
                                                (T*)c->d_pr_cs, c->d_pr_touch);
    return cudaGetLastError();
}

cudaError_t launch_ortho_prepare(Ctx* c, int w, double tol) {
    c->n_launch += 3;
    return c->prec == SSCF_FP64 ? ortho_prepare_t<double>(c, w, tol) : ortho_prepare_t<float>(c, w, tol);
}

template <typename T>
static void fill_args(Ctx* c, SweepArgs& a, int mode, int which) {
    a.mode = mode;
    a.which = which;
    a.n_tiles = c->n_tiles;
    a.n_occ_tiles = c->n_occ_tiles;
    a.n_groups = c->n_groups;
    a.max_cl_groups = c->max_cl_groups;
    a.n_clusters = c->n_clusters;
    a.in_nz = nullptr;
    a.normalise_pass = 1;
    a.gnb_colour = c->d_gnb_colour;
    a.col_lo = 0;
    a.col_hi = c->n_colours;
    a.mol_cluster = c->d_mol_cluster;
    a.cl_g0 = c->d_cl_g0;
    a.cl_ot0 = c->d_cl_ot0;
    a.cl_vt0 = c->d_cl_vt0;
    a.clblk_ptr = c->d_clblk_ptr[mode == 0 ? 0 : 1];
    a.clblk = c->d_clblk[mode == 0 ? 0 : 1];
    a.cap = c->cap;
    a.n_blk = mode == 0 ? c->n_gnb : (int)c->h_ocolour_blk.size();
    a.trunc = mode == 0 ? c->prm.eps : 1e-3 * c->prm.eps;
    a.trunc_f = (float)a.trunc;
    if ((double)a.trunc_f < a.trunc) a.trunc_f = nextafterf(a.trunc_f, INFINITY);
    a.blk = mode == 0 ? c->d_colour_blk : c->d_ocolour_blk;
    a.gnb_row = c->d_gnb_row;
    a.gnb_col = c->d_gnb_col;
    a.group_nmol = c->d_group_nmol;
    a.group_ot0 = c->d_group_ot0;
    a.group_not = c->d_group_not;
    a.group_vt0 = c->d_group_vt0;
    a.group_nvt = c->d_group_nvt;
    a.tile_group = c->d_tile_group;
    a.tile_kind = c->d_tile_kind;
    a.tile_mo0 = c->d_tile_mo0;
    a.tile_nmo = c->d_tile_nmo;
    a.pr_n = c->d_pr_n;
    a.pr_lvl = c->d_pr_lvl;
    a.pr_touch = c->d_pr_touch;
    a.pr_ij = c->d_pr_ij;
    a.pr_cs = c->d_pr_cs;
    a.dsc = c->d_scale;
    a.cl_eta = c->d_cl_eta;
    a.tol = c->ortho_tol;
    a.upd = &c->d_sc->upd[mode == 0 ? 0 : 1];
    a.cci_ptr = c->d_cci_ptr;
    a.cci_row = c->d_cci_row;
    a.cci_slot = c->d_cci_slot;
    a.err = &c->d_sc->err;
}

// The closure of the sweep's colours [col_lo, col_hi) (components over the
// active blocks of those colours); unless it is the first of the pass, a unit
// whose tiles in a row are all flagged zero does not count as held there.
template <typename T>
static cudaError_t closure_t(Ctx* c, int mode, int which, int col_lo, int col_hi, bool first) {
    SweepArgs a;
    fill_args<T>(c, a, mode, which);
    const int in = c->cur, out = 1 - c->cur;
    a.in_nt = c->d_c_nt[in];
    a.in_tile = c->d_c_tile[in];
    a.in_val = c->d_c_val[in];
    a.out_nt = c->d_c_nt[out];
    a.out_tile = c->d_c_tile[out];
    a.out_val = c->d_c_val[out];
    a.out_nz = c->d_c_nz[out];
    a.unit_lab = c->d_unit_lab;
    a.in_nz = first ? nullptr : c->d_c_nz[in];
    a.normalise_pass = first ? 1 : 0;
    a.col_lo = col_lo;
    a.col_hi = col_hi;
    const size_t smem = closure_smem_bytes(c);
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_closure<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    a.lab_start = c->d_lab_start;
    a.lab_cnt = c->d_lab_cnt;
    a.lab_mem = c->d_lab_mem;
    const size_t lsmem = closure_labels_smem_bytes(c);
    if (lsmem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(k_closure_labels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem);
    if (e != cudaSuccess) return e;
    k_closure_labels<<<c->n_clusters, 1024, lsmem, c->stream>>>(a, c->d_unit_lab);
    k_closure<T><<<c->n_mol, 256, smem, c->stream>>>(a);
    c->cur = out;
    return cudaGetLastError();
}

template <typename T, int MODE, int NT, int PCAP>
static cudaError_t apply_mode_t(Ctx* c, int which, int col_lo, int col_hi) {
    SweepArgs a;
    fill_args<T>(c, a, MODE, which);
    a.in_nt = a.out_nt = c->d_c_nt[c->cur];
    a.in_tile = a.out_tile = c->d_c_tile[c->cur];
    a.in_val = a.out_val = c->d_c_val[c->cur];
    a.out_nz = c->d_c_nz[c->cur];
    a.col_nz = c->d_c_cnz;
    const size_t smem = (size_t)NT * 16 * apply_nrp<T>() * sizeof(T) + (size_t)2 * PCAP * sizeof(T) + (size_t)PCAP * 4;
    cudaError_t e = cudaFuncSetAttribute(k_apply_colour<T, MODE, NT, PCAP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const std::vector<int>& ptr = MODE == 0 ? c->h_colour_ptr : c->h_ocolour_ptr;
    constexpr int CH = ApplyShape<T>::chunk;
    const int gx = (c->n_mol + CH - 1) / CH;
    // FP32 rotations and occupied passes: blocks between full groups take the register-resident kernel
    const bool full = std::is_same<T, float>::value && (MODE == 0 || which == 1) && c->apply_variant != 1;
    if (full) {
        e = cudaFuncSetAttribute(k_apply_full<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)full_apply_smem<MODE>());
        if (e != cudaSuccess) return e;
    }
    const std::vector<int>& nfull = MODE == 0 ? c->h_colour_nfull : c->h_ocolour_nfull;
    // row chunks per block in x: enough CTAs to fill the GPU a few times over,
    // each looping over its chunks with one coefficient table
    static int full_occ[2] = {0, 0};
    if (full && full_occ[MODE] == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&full_occ[MODE], k_apply_full<MODE>, kFullThreads,
                                                              full_apply_smem<MODE>());
        if (e != cudaSuccess) return e;
        full_occ[MODE] = std::max(full_occ[MODE], 1);
    }
    const int chunks = (c->n_mol + kFullCH - 1) / kFullCH;
    k_flags_by_column<<<c->n_tiles, 256, 0, c->stream>>>(c->cap, c->d_cci_ptr, c->d_cci_row, c->d_cci_slot,
                                                         a.out_nz, a.col_nz);
    c->n_launch += 1;
    if (full && a.n_blk > 0) {
        a.blk_info = (const int4*)c->d_blk_info;
        k_block_info<MODE><<<(a.n_blk + 127) / 128, 128, 0, c->stream>>>(a, a.n_blk, (int4*)c->d_blk_info);
        c->n_launch += 1;
    }
    for (int col = col_lo; col < col_hi; ++col) {
        const int nf = full ? nfull[col] : 0;
        if (nf > 0) {
            // variant 2: one CTA takes all row chunks of its block (the longest
            // collection of row pairs; same results)
            const int gxf = c->apply_variant == 2
                                ? 1
                                : std::min(chunks, std::max(1, (kFullWaves[MODE] * c->n_sm * full_occ[MODE]) /
                                                                   std::max(nf, 1) + 1));
            k_apply_full<MODE><<<dim3(gxf, nf), kFullThreads, full_apply_smem<MODE>(), c->stream>>>(a, ptr[col]);
            c->n_launch += 1;
        }
        const int nb = ptr[col + 1] - ptr[col] - nf;
        if (nb == 0) continue;
        dim3 grid(gx, nb);
        k_apply_colour<T, MODE, NT, PCAP><<<grid, apply_threads<T>(), smem, c->stream>>>(a, ptr[col] + nf);
        c->n_launch += 1;
    }
    return cudaGetLastError();
}

// side tiles and pair capacity per pass: rotations 2 occupied + 1 virtual
// tiles, 32 x 16 pairs; occupied passes 2 + 2 tiles, 32 x 32 pairs; passes over
// all MOs 3 + 3 tiles, 48 x 48 pairs
template <typename T>
static cudaError_t apply_t(Ctx* c, int mode, int which, int col_lo, int col_hi) {
    if (mode == 0) return apply_mode_t<T, 0, 3, kRotCap>(c, which, col_lo, col_hi);
    if (which == 1) return apply_mode_t<T, 1, 4, 32 * 32>(c, which, col_lo, col_hi);
    return apply_mode_t<T, 1, 6, kOrthoCap>(c, which, col_lo, col_hi);
}

cudaError_t launch_closure(Ctx* c, int mode, int which, int col_lo, int col_hi, bool first) {
    c->n_launch += 2;
    if (col_hi < 0) col_hi = c->n_colours;
    return c->prec == SSCF_FP64 ? closure_t<double>(c, mode, which, col_lo, col_hi, first)
                                : closure_t<float>(c, mode, which, col_lo, col_hi, first);
}

cudaError_t launch_apply(Ctx* c, int mode, int which, int col_lo, int col_hi) {
    if (col_hi < 0) col_hi = c->n_colours;
    return c->prec == SSCF_FP64 ? apply_t<double>(c, mode, which, col_lo, col_hi)
                                : apply_t<float>(c, mode, which, col_lo, col_hi);
}

cudaError_t launch_compact(Ctx* c) {
    c->n_launch += 1;
    const int in = c->cur, out = 1 - c->cur;
    if (c->prec == SSCF_FP64)
        k_compact<double><<<c->n_mol, 256, 0, c->stream>>>(c->cap, c->d_c_nt[in], c->d_c_tile[in],
                                                           (const double*)c->d_c_val[in], c->d_c_nt[out],
                                                           c->d_c_tile[out], (double*)c->d_c_val[out], &c->d_sc->err);
    else
        k_compact<float><<<c->n_mol, 256, 0, c->stream>>>(c->cap, c->d_c_nt[in], c->d_c_tile[in],
                                                          (const float*)c->d_c_val[in], c->d_c_nt[out],
                                                          c->d_c_tile[out], (float*)c->d_c_val[out], &c->d_sc->err);
    c->cur = out;
    return cudaGetLastError();
}

}  // namespace sscf
