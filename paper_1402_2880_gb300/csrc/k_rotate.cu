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

#include "sscf_internal.h"

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
// rotation candidates: count |F_ij| >= tau (F_ij != 0) and the largest |F|
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_rot_stats(int n_gnb, const int* __restrict__ gnb_row, const int* __restrict__ gnb_col,
                            const int* __restrict__ group_nmol, const int* __restrict__ group_nvt,
                            const int* __restrict__ blk_tp0, const T* __restrict__ F, double tau,
                            DeviceScalars* sc) {
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
        if (cnt) atomicAdd(&sc->cand, (unsigned long long)cnt);
        atomic_max_pos(&sc->max_fov, mx);
    }
}

// one radix-select pass over the candidate keys (8 bits, most significant first)
template <typename T>
__global__ void k_rot_hist(int shift, unsigned long long kmax, int n_gnb, const int* __restrict__ gnb_row,
                           const int* __restrict__ gnb_col, const int* __restrict__ group_nmol,
                           const int* __restrict__ group_nvt, const int* __restrict__ blk_tp0,
                           const T* __restrict__ F, double tau, DeviceScalars* sc) {
    if (sc->cand <= kmax) return;
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long prefix = sc->sel_prefix, mask = sc->sel_mask;
    for (int e = blockIdx.x; e < n_gnb; e += gridDim.x) {
        const int A = gnb_row[e], B = gnb_col[e];
        const int no = 4 * group_nmol[A], nv = 2 * group_nmol[B], nvt = group_nvt[B];
        for (int p = threadIdx.x; p < no * nv; p += blockDim.x) {
            const int i = p / nv, j = p % nv;
            const int tp = blk_tp0[e] + (i >> 4) * nvt + (j >> 4);
            const double f = fabs((double)F[(size_t)tp * 256 + (i & 15) * 16 + (j & 15)]);
            if (!(f >= tau && f > 0.0)) continue;
            const unsigned long long k = dkey(f);
            if ((k & mask) != prefix) continue;
            atomicAdd(&h[(k >> shift) & 255ull], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&sc->hist[i], (unsigned long long)h[i]);
}

__global__ void k_rot_pick(int shift, unsigned long long kmax, DeviceScalars* sc) {
    if (sc->cand <= kmax) return;
    if (shift == 56) {
        sc->sel_k = kmax;
    }
    unsigned long long k = sc->sel_k, cum = 0;
    int b = 255;
    for (; b > 0; --b) {
        if (cum + sc->hist[b] >= k) break;
        cum += sc->hist[b];
    }
    sc->sel_prefix |= (unsigned long long)b << shift;
    sc->sel_mask |= 255ull << shift;
    sc->sel_k = k - cum;
    for (int i = 0; i < 256; ++i) sc->hist[i] = 0;
}

__global__ void k_rot_threshold(unsigned long long kmax, double tau, DeviceScalars* sc) {
    sc->thr_key = sc->cand > kmax ? sc->sel_prefix : 0ull;
}

// per block: kept pairs sorted by (in-block colour, i_loc) with Jacobi angles
// p = (F_ii - F_jj) / (2 F_ij), t = 1/(p + sgn(p) sqrt(1 + p^2)),
// c = 1/sqrt(1 + t^2), s = t c in FP64 (sgn(0) = +1)
template <typename T>
__global__ void k_rot_lists(int n_gnb, const int* __restrict__ gnb_row, const int* __restrict__ gnb_col,
                            const int* __restrict__ group_nmol, const int* __restrict__ group_nvt,
                            const int* __restrict__ group_occ0_mo, const int* __restrict__ group_virt0_mo,
                            const int* __restrict__ blk_tp0, const T* __restrict__ F,
                            const double* __restrict__ Fd, double tau, DeviceScalars* sc, int* __restrict__ pr_n,
                            int* __restrict__ pr_lvl, uint16_t* __restrict__ pr_ij, T* __restrict__ pr_cs,
                            int* __restrict__ pr_touch) {
    __shared__ unsigned char keep[32 * 16];
    __shared__ int cnt[kMaxSub + 1];
    const int e = blockIdx.x;
    const int A = gnb_row[e], B = gnb_col[e];
    const int no = 4 * group_nmol[A], nv = 2 * group_nmol[B], nvt = group_nvt[B];
    const int nsub = max(no, nv);
    const unsigned long long thr = sc->thr_key;
    for (int p = threadIdx.x; p < 32 * 16; p += blockDim.x) {
        int i = p >> 4, j = p & 15;
        unsigned char kp = 0;
        if (i < no && j < nv) {
            const int tp = blk_tp0[e] + (i >> 4) * nvt + (j >> 4);
            const double f = fabs((double)F[(size_t)tp * 256 + (i & 15) * 16 + (j & 15)]);
            kp = (f >= tau && f > 0.0 && dkey(f) >= thr) ? 1 : 0;
        }
        keep[p] = kp;
    }
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
        int touch = 0;
        for (int i = 0; i < no; ++i)
            for (int j = 0; j < nv; ++j)
                if (keep[i * 16 + j]) touch |= (1 << (i >> 4)) | (1 << (3 + (j >> 4)));
        pr_touch[e] = touch;
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
                            const T* __restrict__ sig, const double* __restrict__ dsc, DeviceScalars* sc) {
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
    if ((threadIdx.x & 31) == 0) atomic_max_pos(&sc->eta, mx);
}

template <typename T>
__global__ void k_ortho_lists(int w, double tol, const int* __restrict__ oblk, const int* __restrict__ gnb_row,
                              const int* __restrict__ gnb_col, const int* __restrict__ group_nmol,
                              const int* __restrict__ group_not, const int* __restrict__ occ0,
                              const int* __restrict__ virt0, const int* __restrict__ blk_tp,
                              const T* __restrict__ sig, const double* __restrict__ dsc, DeviceScalars* sc,
                              int* __restrict__ pr_n, int* __restrict__ pr_lvl, uint16_t* __restrict__ pr_ij,
                              T* __restrict__ pr_cs, int* __restrict__ pr_touch) {
    __shared__ unsigned char keep[48 * 48];
    __shared__ int cnt[kMaxSub + 1];
    const int e = oblk[blockIdx.x];
    const int A = gnb_row[e], B = gnb_col[e];
    const int noA = 4 * group_nmol[A], noB = 4 * group_nmol[B];
    const int nA = w == 1 ? noA : 6 * group_nmol[A], nB = w == 1 ? noB : 6 * group_nmol[B];
    const bool same = A == B;
    const int nsub = max(nA, nB);
    const double eta = sc->eta;
    const bool active = !(eta < tol);
    const double cut = 1e-3 * eta;
    for (int p = threadIdx.x; p < 48 * 48; p += blockDim.x) {
        const int i = p / 48, j = p % 48;
        unsigned char kp = 0;
        if (active && i < nA && j < nB && !(same && j <= i)) {
            int ia, ci, ib, cj;
            side_pos(i, noA, group_not[A], ia, ci);
            side_pos(j, noB, group_not[B], ib, cj);
            const double di = dsc[pass_mo(i, noA, occ0, virt0, A)], dj = dsc[pass_mo(j, noB, occ0, virt0, B)];
            kp = fabs(sig_hat(sig, blk_tp, e, same, ia, ib, ci, cj, di, dj)) >= cut ? 1 : 0;
        }
        keep[p] = kp;
    }
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
        int touch = 0;
        for (int i = 0; i < nA; ++i)
            for (int j = 0; j < nB; ++j)
                if (keep[i * 48 + j]) {
                    int ia, ci, ib, cj;
                    side_pos(i, noA, group_not[A], ia, ci);
                    side_pos(j, noB, group_not[B], ib, cj);
                    touch |= (1 << ia) | (1 << (3 + ib));
                }
        pr_touch[e] = touch;
    }
    __syncthreads();
    if ((int)threadIdx.x < nsub) {
        const int s = threadIdx.x;
        int pos = pr_lvl[(size_t)e * (kMaxSub + 1) + s];
        for (int i = 0; i < nA; ++i) {
            int j = ((s - i) % nsub + nsub) % nsub;
            if (!(j < nB && keep[i * 48 + j])) continue;
            int ia, ci, ib, cj;
            side_pos(i, noA, group_not[A], ia, ci);
            side_pos(j, noB, group_not[B], ib, cj);
            const double di = dsc[pass_mo(i, noA, occ0, virt0, A)], dj = dsc[pass_mo(j, noB, occ0, virt0, B)];
            const double sh = sig_hat(sig, blk_tp, e, same, ia, ib, ci, cj, di, dj);
            const size_t q = (size_t)e * kOrthoCap + pos;
            pr_ij[q] = (uint16_t)(i | (j << 8));
            pr_cs[2 * q] = (T)__dmul_rn(0.5, sh);
            pr_cs[2 * q + 1] = (T)0;
            ++pos;
        }
    }
}

// --------------------------------------------------------------------------
// row-local application of a whole sweep
// --------------------------------------------------------------------------
struct ApplyArgs {
    int mode;        // 0 rotations (occupied A x virtual B), 1 combinations
    int which;       // combinations: 0 all MOs, 1 occupied
    int n_tiles, n_occ_tiles, n_groups, cap, n_colours;
    double trunc;
    const int* colour_ptr;
    const int* colour_blk;
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
    const uint16_t* pr_ij;
    const void* pr_cs;
    const int* pr_touch;
    const double* dsc;    // mode 1: divide the pass's MOs by d_i first
    const int* in_nt;
    const int* in_tile;
    const void* in_val;
    int* out_nt;
    int* out_tile;
    void* out_val;
    unsigned* err;
};

constexpr int kApplyWarps = 8;

template <typename T>
__global__ void __launch_bounds__(kApplyWarps * 32) k_apply(ApplyArgs a) {
    extern __shared__ unsigned char smraw[];
    const int cap = a.cap;
    int np2 = 1;
    while (np2 < cap) np2 <<= 1;
    T* vals = (T*)smraw;                                        // cap * 16
    unsigned* keys = (unsigned*)(vals + (size_t)cap * 16);      // np2 (tile << 16 | slot)
    short* map = (short*)(keys + np2);                          // n_tiles
    unsigned* pres = (unsigned*)(map + ((a.n_tiles + 1) & ~1));  // 2 * ceil(G/32)
    __shared__ int s_n, s_abort;
    const int gw = (a.n_groups + 31) >> 5;
    const int r = blockIdx.x / 6, krow = blockIdx.x % 6;
    const T* inv = (const T*)a.in_val;
    for (int i = threadIdx.x; i < a.n_tiles; i += blockDim.x) map[i] = -1;
    for (int i = threadIdx.x; i < 2 * gw; i += blockDim.x) pres[i] = 0u;
    if (threadIdx.x == 0) {
        s_n = a.in_nt[r];
        s_abort = 0;
    }
    __syncthreads();
    const int n0 = s_n;
    for (int s = threadIdx.x; s < n0; s += blockDim.x) {
        const int t = a.in_tile[(size_t)r * cap + s];
        map[t] = (short)s;
        const int g = a.tile_group[t];
        atomicOr(&pres[a.tile_kind[t] * gw + (g >> 5)], 1u << (g & 31));
    }
    for (int idx = threadIdx.x; idx < n0 * 16; idx += blockDim.x) {
        const int s = idx >> 4, c = idx & 15;
        T v = inv[(((size_t)r * cap + s) * 6 + krow) * 16 + c];
        if (a.mode == 1) {
            const int t = a.in_tile[(size_t)r * cap + s];
            const bool in_pass = a.which == 0 || a.tile_kind[t] == 0;
            if (in_pass && c < a.tile_nmo[t]) v = (T)((double)v / a.dsc[a.tile_mo0[t] + c]);
        }
        vals[idx] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T* cs = (const T*)a.pr_cs;
    for (int col = 0; col < a.n_colours; ++col) {
        const int b0 = a.colour_ptr[col], b1 = a.colour_ptr[col + 1];
        for (int jb = b0 + warp; jb < b1; jb += kApplyWarps) {
            const int e = a.colour_blk[jb];
            const int np = a.pr_n[e];
            if (np == 0) continue;
            const int A = a.gnb_row[e], B = a.gnb_col[e];
            const int touch = a.pr_touch[e];
            // side tiles: rotations: A occ | B virt; combinations: occ (+ virt) of A | of B
            int st[6];
            int nsa = 0, nsb = 0;
            for (int i = 0; i < a.group_not[A]; ++i) st[nsa++] = a.group_ot0[A] + i;
            if (a.mode == 1 && a.which == 0)
                for (int i = 0; i < a.group_nvt[A]; ++i) st[nsa++] = a.group_vt0[A] + i;
            if (a.mode == 1) {
                for (int i = 0; i < a.group_not[B]; ++i) st[3 + nsb++] = a.group_ot0[B] + i;
                if (a.which == 0)
                    for (int i = 0; i < a.group_nvt[B]; ++i) st[3 + nsb++] = a.group_vt0[B] + i;
            } else {
                for (int i = 0; i < a.group_nvt[B]; ++i) st[3 + nsb++] = a.group_vt0[B] + i;
            }
            bool relevant = false;
            for (int i = 0; i < 6; ++i) {
                const bool in_side = i < 3 ? i < nsa : (i - 3) < nsb;
                if (in_side && ((touch >> i) & 1) && map[st[i]] >= 0) relevant = true;
            }
            if (!relevant) continue;
            int slot[6];
            if (lane == 0) {
                for (int i = 0; i < 6; ++i) {
                    slot[i] = -1;
                    const bool in_side = i < 3 ? i < nsa : (i - 3) < nsb;
                    if (!in_side || !((touch >> i) & 1)) continue;
                    const int t = st[i];
                    int s = map[t];
                    if (s < 0) {
                        s = atomicAdd(&s_n, 1);
                        if (s >= cap) {
                            atomicOr(a.err, kErrCapacity);
                            s_abort = 1;
                            s = -1;
                        } else {
                            for (int c = 0; c < 16; ++c) vals[(size_t)s * 16 + c] = (T)0;
                            map[t] = (short)s;
                            const int g = a.tile_group[t];
                            atomicOr(&pres[a.tile_kind[t] * gw + (g >> 5)], 1u << (g & 31));
                        }
                    }
                    slot[i] = s;
                }
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) slot[i] = __shfl_sync(0xffffffffu, slot[i], 0);
            __syncwarp();
            bool bad = false;
            for (int i = 0; i < 6; ++i) {
                const bool in_side = i < 3 ? i < nsa : (i - 3) < nsb;
                if (in_side && ((touch >> i) & 1) && slot[i] < 0) bad = true;
            }
            if (bad) continue;
            const int noA = 4 * a.group_nmol[A], noB = 4 * a.group_nmol[B];
            const int* lvl = a.pr_lvl + (size_t)e * (kMaxSub + 1);
            for (int sub = 0; sub < kMaxSub; ++sub) {
                const int q0 = lvl[sub], q1 = lvl[sub + 1];
                if (q0 == np) break;
                for (int q = q0 + lane; q < q1; q += 32) {
                    const size_t qq = (size_t)e * kOrthoCap + q;
                    const unsigned ij = a.pr_ij[qq];
                    const int il = ij & 255, jl = ij >> 8;
                    int ta, ca, tb, cb;
                    if (a.mode == 0) {
                        ta = il >> 4;
                        ca = il & 15;
                        tb = 3 + (jl >> 4);
                        cb = jl & 15;
                    } else {
                        side_pos(il, noA, a.group_not[A], ta, ca);
                        side_pos(jl, noB, a.group_not[B], tb, cb);
                        tb += 3;
                    }
                    T* pi = vals + (size_t)slot[ta] * 16 + ca;
                    T* pj = vals + (size_t)slot[tb] * 16 + cb;
                    const T x = *pi, y = *pj;
                    T xn, yn;
                    if (a.mode == 0) {
                        const T c = cs[2 * qq], s = cs[2 * qq + 1];
                        xn = c * x + s * y;
                        yn = -s * x + c * y;
                    } else {
                        const T h = cs[2 * qq];
                        xn = x - h * y;
                        yn = y - h * x;
                    }
                    *pi = fabs((double)xn) < a.trunc ? (T)0 : xn;
                    *pj = fabs((double)yn) < a.trunc ? (T)0 : yn;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_abort) return;
    }
    // write back, tiles sorted by id
    const int n = s_n;
    for (int i = threadIdx.x; i < np2; i += blockDim.x) keys[i] = 0xffffffffu;
    __syncthreads();
    for (int t = threadIdx.x; t < a.n_tiles; t += blockDim.x)
        if (map[t] >= 0) keys[map[t]] = ((unsigned)t << 16) | (unsigned)map[t];
    __syncthreads();
    for (int k = 2; k <= np2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & k) == 0;
                    unsigned x = keys[i], y = keys[l];
                    if ((x > y) == up) {
                        keys[i] = y;
                        keys[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    T* outv = (T*)a.out_val;
    if (krow == 0) {
        for (int s = threadIdx.x; s < n; s += blockDim.x) a.out_tile[(size_t)r * cap + s] = (int)(keys[s] >> 16);
        if (threadIdx.x == 0) a.out_nt[r] = n;
    }
    for (int idx = threadIdx.x; idx < n * 16; idx += blockDim.x) {
        const int s = idx >> 4, c = idx & 15;
        const int src = keys[s] & 0xffffu;
        outv[(((size_t)r * cap + s) * 6 + krow) * 16 + c] = vals[(size_t)src * 16 + c];
    }
}

// drop tiles whose 6x16 values are all zero; in -> out
template <typename T>
__global__ void k_compact(int cap, const int* __restrict__ in_nt, const int* __restrict__ in_tile,
                          const T* __restrict__ in_val, int* __restrict__ out_nt, int* __restrict__ out_tile,
                          T* __restrict__ out_val) {
    __shared__ int wcnt[32];
    __shared__ int s_base;
    const int r = blockIdx.x;
    const int n = in_nt[r];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    // process in chunks of nwarps tiles, one warp per tile, order preserved
    for (int s0 = 0; s0 < n; s0 += nwarps) {
        const int s = s0 + warp;
        bool nz = false;
        if (s < n) {
            const T* v = in_val + ((size_t)r * cap + s) * kTileVals;
            for (int i = lane; i < kTileVals; i += 32) nz |= (v[i] != (T)0);
        }
        nz = __any_sync(0xffffffffu, nz);
        if (lane == 0) wcnt[warp] = (s < n && nz) ? 1 : 0;
        __syncthreads();
        int pos = s_base;
        for (int w = 0; w < warp; ++w) pos += wcnt[w];
        if (s < n && nz) {
            const T* v = in_val + ((size_t)r * cap + s) * kTileVals;
            T* o = out_val + ((size_t)r * cap + pos) * kTileVals;
            for (int i = lane; i < kTileVals; i += 32) o[i] = v[i];
            if (lane == 0) out_tile[(size_t)r * cap + pos] = in_tile[(size_t)r * cap + s];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nwarps; ++w) tot += wcnt[w];
            s_base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out_nt[r] = s_base;
}

}  // namespace

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
template <typename T>
static cudaError_t select_rot_t(Ctx* c) {
    const double tau = c->prm.eps;
    const unsigned long long kmax = (unsigned long long)(c->prm.rot_cap_factor * (double)c->n_occ);
    k_rot_stats<T><<<c->n_gnb, 256, 0, c->stream>>>(c->n_gnb, c->d_gnb_row, c->d_gnb_col, c->d_group_nmol,
                                                    c->d_group_nvt, c->d_rot_blk_tp0, (const T*)c->d_F, tau, c->d_sc);
    const int hb = std::min(c->n_gnb, 1024);
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_rot_hist<T><<<hb, 256, 0, c->stream>>>(shift, kmax, c->n_gnb, c->d_gnb_row, c->d_gnb_col, c->d_group_nmol,
                                                 c->d_group_nvt, c->d_rot_blk_tp0, (const T*)c->d_F, tau, c->d_sc);
        k_rot_pick<<<1, 1, 0, c->stream>>>(shift, kmax, c->d_sc);
    }
    k_rot_threshold<<<1, 1, 0, c->stream>>>(kmax, tau, c->d_sc);
    k_rot_lists<T><<<c->n_gnb, 128, 0, c->stream>>>(
        c->n_gnb, c->d_gnb_row, c->d_gnb_col, c->d_group_nmol, c->d_group_nvt, c->d_group_occ0_mo,
        c->d_group_virt0_mo, c->d_rot_blk_tp0, (const T*)c->d_F, c->d_Fd, tau, c->d_sc, c->d_pr_n, c->d_pr_lvl,
        c->d_pr_ij, (T*)c->d_pr_cs, c->d_pr_touch);
    return cudaGetLastError();
}

cudaError_t launch_select_rot(Ctx* c) {
    return c->prec == SSCF_FP64 ? select_rot_t<double>(c) : select_rot_t<float>(c);
}

template <typename T>
static cudaError_t ortho_prepare_t(Ctx* c, int w, double tol) {
    const int t_hi = w == 1 ? c->n_occ_tiles : c->n_tiles;
    k_ortho_scale<T><<<(t_hi * 16 + 255) / 256, 256, 0, c->stream>>>(
        w, 0, t_hi, c->d_tile_group, c->d_tile_kind, c->d_tile_nmo, c->d_tile_mo0, c->d_group_ot0, c->d_group_not,
        c->d_group_vt0, c->d_self_blk, c->d_ort_blk_tp[w], (const T*)c->d_sig, c->d_scale, &c->d_sc->err);
    const int nob = (int)c->h_ocolour_blk.size();
    k_ortho_eta<T><<<nob, 256, 0, c->stream>>>(w, c->d_ocolour_blk, nob, c->d_gnb_row, c->d_gnb_col,
                                              c->d_group_nmol, c->d_group_not, c->d_group_occ0_mo,
                                              c->d_group_virt0_mo, c->d_ort_blk_tp[w], (const T*)c->d_sig,
                                              c->d_scale, c->d_sc);
    k_ortho_lists<T><<<nob, 128, 0, c->stream>>>(w, tol, c->d_ocolour_blk, c->d_gnb_row, c->d_gnb_col,
                                                c->d_group_nmol, c->d_group_not, c->d_group_occ0_mo,
                                                c->d_group_virt0_mo, c->d_ort_blk_tp[w], (const T*)c->d_sig,
                                                c->d_scale, c->d_sc, c->d_pr_n, c->d_pr_lvl, c->d_pr_ij,
                                                (T*)c->d_pr_cs, c->d_pr_touch);
    return cudaGetLastError();
}

cudaError_t launch_ortho_prepare(Ctx* c, int w, double tol) {
    return c->prec == SSCF_FP64 ? ortho_prepare_t<double>(c, w, tol) : ortho_prepare_t<float>(c, w, tol);
}

size_t apply_smem_bytes(const Ctx* c) {
    int np2 = 1;
    while (np2 < c->cap) np2 <<= 1;
    size_t b = (size_t)c->cap * 16 * c->tsize + (size_t)np2 * 4 + (size_t)((c->n_tiles + 1) & ~1) * 2 +
               (size_t)2 * ((c->n_groups + 31) / 32) * 4;
    return (b + 15) & ~(size_t)15;
}

template <typename T>
static cudaError_t apply_t(Ctx* c, int mode, int which) {
    const size_t smem = apply_smem_bytes(c);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ApplyArgs a;
    a.mode = mode;
    a.which = which;
    a.n_tiles = c->n_tiles;
    a.n_occ_tiles = c->n_occ_tiles;
    a.n_groups = c->n_groups;
    a.cap = c->cap;
    a.n_colours = c->n_colours;
    a.trunc = mode == 0 ? c->prm.eps : 1e-3 * c->prm.eps;
    a.colour_ptr = mode == 0 ? c->d_colour_ptr : c->d_ocolour_ptr;
    a.colour_blk = mode == 0 ? c->d_colour_blk : c->d_ocolour_blk;
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
    a.pr_ij = c->d_pr_ij;
    a.pr_cs = c->d_pr_cs;
    a.pr_touch = c->d_pr_touch;
    a.dsc = c->d_scale;
    const int in = c->cur, out = 1 - c->cur;
    a.in_nt = c->d_c_nt[in];
    a.in_tile = c->d_c_tile[in];
    a.in_val = c->d_c_val[in];
    a.out_nt = c->d_c_nt[out];
    a.out_tile = c->d_c_tile[out];
    a.out_val = c->d_c_val[out];
    a.err = &c->d_sc->err;
    k_apply<T><<<c->n_mol * 6, kApplyWarps * 32, smem, c->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_apply(Ctx* c, int mode, int which) {
    return c->prec == SSCF_FP64 ? apply_t<double>(c, mode, which) : apply_t<float>(c, mode, which);
}

cudaError_t launch_compact(Ctx* c) {
    const int in = 1 - c->cur, out = c->cur;
    if (c->prec == SSCF_FP64)
        k_compact<double><<<c->n_mol, 256, 0, c->stream>>>(c->cap, c->d_c_nt[in], c->d_c_tile[in],
                                                           (const double*)c->d_c_val[in], c->d_c_nt[out],
                                                           c->d_c_tile[out], (double*)c->d_c_val[out]);
    else
        k_compact<float><<<c->n_mol, 256, 0, c->stream>>>(c->cap, c->d_c_nt[in], c->d_c_tile[in],
                                                          (const float*)c->d_c_val[in], c->d_c_nt[out],
                                                          c->d_c_tile[out], (float*)c->d_c_val[out]);
    return cudaGetLastError();
}

}  // namespace sscf
