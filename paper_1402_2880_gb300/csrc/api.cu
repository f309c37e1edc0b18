// C-ABI of libsscf: context creation (step I structure on the host), device
// allocation, and the order of kernel launches of every step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <new>

#include "sscf_internal.h"

using namespace sscf;

namespace {

sscf_alloc_fn g_alloc = nullptr;
sscf_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) {                                          \
            fprintf(stderr, "libsscf: %s failed: %s (%s:%d)\n", #call,     \
                    cudaGetErrorString(e_), __FILE__, __LINE__);          \
            return SSCF_ERR_CUDA;                                         \
        }                                                                 \
    } while (0)

#define CKS(call)                              \
    do {                                       \
        int s_ = (call);                       \
        if (s_ != SSCF_OK) return s_;          \
    } while (0)

// Squared distance evaluated as (dx*dx + dy*dy) + dz*dz. The library is
// compiled with -ffp-contract=off so that no product is fused into the sums:
// neighbour decisions are then bit-identical to any other IEEE evaluation of
// the same expression.
inline double dist2(const double* a, const double* b) {
    double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    double xx = dx * dx, yy = dy * dy, zz = dz * dz;
    double s = xx + yy;
    return s + zz;
}

struct CellGrid {
    double lo[3], h;
    int n[3];
    std::vector<int> head, next;
    void build(const std::vector<double>& pts, int npts, double cell) {
        for (int d = 0; d < 3; ++d) lo[d] = 1e300;
        double hi[3] = {-1e300, -1e300, -1e300};
        for (int i = 0; i < npts; ++i)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], pts[3 * i + d]);
                hi[d] = std::max(hi[d], pts[3 * i + d]);
            }
        h = cell;
        for (int d = 0; d < 3; ++d) n[d] = std::max(1, (int)std::floor((hi[d] - lo[d]) / h) + 1);
        head.assign((size_t)n[0] * n[1] * n[2], -1);
        next.assign(npts, -1);
        for (int i = 0; i < npts; ++i) {
            int c = cell_of(&pts[3 * i]);
            next[i] = head[c];
            head[c] = i;
        }
    }
    int coord(const double* p, int d) const {
        int k = (int)std::floor((p[d] - lo[d]) / h);
        return std::min(std::max(k, 0), n[d] - 1);
    }
    int cell_of(const double* p) const {
        return coord(p, 0) + n[0] * (coord(p, 1) + n[1] * coord(p, 2));
    }
};

int build_structure(Ctx& c, const sscf_system* sys) {
    const int nA = c.n_atoms, nM = c.n_mol;
    const double* X = c.h_xyz.data();
    // ---- molecule pairs with an atom pair within r_cut (plus (m, m)) ----
    std::vector<double> ox(3 * nM);
    std::vector<double> rad(nM, 0.0);
    double rmax = 0.0;
    for (int m = 0; m < nM; ++m) {
        for (int d = 0; d < 3; ++d) ox[3 * m + d] = X[3 * (3 * m) + d];
        for (int k = 1; k < 3; ++k) rad[m] = std::max(rad[m], std::sqrt(dist2(&X[9 * m], &X[9 * m + 3 * k])));
        rmax = std::max(rmax, rad[m]);
    }
    const double rc2 = c.prm.r_cut * c.prm.r_cut;
    std::vector<std::vector<int>> nbm(nM);
    // clusters never couple: one cell grid per cluster (molecules of a cluster are consecutive)
    for (int k = 0; k < c.n_clusters; ++k) {
        const int m0 = c.h_cl_mol0[k], nk = c.h_cl_nmol[k];
        std::vector<double> oxk(ox.begin() + 3 * (size_t)m0, ox.begin() + 3 * (size_t)(m0 + nk));
        CellGrid grid;
        grid.build(oxk, nk, c.prm.r_cut + 2.0 * rmax + 1e-9);
        for (int m = m0; m < m0 + nk; ++m) {
            int cx = grid.coord(&ox[3 * m], 0), cy = grid.coord(&ox[3 * m], 1), cz = grid.coord(&ox[3 * m], 2);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int x = cx + dx, y = cy + dy, z = cz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= grid.n[0] || y >= grid.n[1] || z >= grid.n[2]) continue;
                        for (int nl = grid.head[x + grid.n[0] * (y + grid.n[1] * z)]; nl >= 0; nl = grid.next[nl]) {
                            const int n = m0 + nl;
                            bool hit = (n == m);
                            for (int a = 0; a < 3 && !hit; ++a)
                                for (int b = 0; b < 3 && !hit; ++b)
                                    if (dist2(&X[3 * (3 * m + a)], &X[3 * (3 * n + b)]) <= rc2) hit = true;
                            if (hit) nbm[m].push_back(n);
                        }
                    }
            std::sort(nbm[m].begin(), nbm[m].end());
        }
    }
    c.h_mp_ptr.assign(nM + 1, 0);
    for (int m = 0; m < nM; ++m) c.h_mp_ptr[m + 1] = c.h_mp_ptr[m] + (int)nbm[m].size();
    c.n_mp = c.h_mp_ptr[nM];
    c.h_mp_col.resize(c.n_mp);
    for (int m = 0; m < nM; ++m) std::copy(nbm[m].begin(), nbm[m].end(), c.h_mp_col.begin() + c.h_mp_ptr[m]);

    // ---- groups ----
    const int G = c.n_groups;
    std::vector<std::vector<int>> mols(G);
    for (int m = 0; m < nM; ++m) mols[c.h_mol_group[m]].push_back(m);
    c.h_mol_local.assign(nM, 0);
    c.h_group_nmol.assign(G, 0);
    c.h_group_occ0.assign(G, 0);
    c.h_group_virt0.assign(G, 0);
    c.h_group_ot0.assign(G, 0);
    c.h_group_not.assign(G, 0);
    c.h_group_vt0.assign(G, 0);
    c.h_group_nvt.assign(G, 0);
    int o = 0, v = c.n_occ, ot = 0;
    for (int g = 0; g < G; ++g) {
        if (mols[g].empty() || mols[g].size() > (size_t)kMaxMolPerGroup) return SSCF_ERR_INVALID_ARG;
        for (int m : mols[g])
            if (c.h_mol_cluster[m] != c.h_mol_cluster[mols[g][0]]) return SSCF_ERR_INVALID_ARG;
        if (g > 0 && c.h_mol_cluster[mols[g][0]] < c.h_mol_cluster[mols[g - 1][0]]) return SSCF_ERR_INVALID_ARG;
        for (size_t k = 0; k < mols[g].size(); ++k) c.h_mol_local[mols[g][k]] = (int)k;
        int nm = (int)mols[g].size();
        c.h_group_nmol[g] = nm;
        c.h_group_occ0[g] = o;
        c.h_group_virt0[g] = v;
        o += 4 * nm;
        v += 2 * nm;
        c.h_group_ot0[g] = ot;
        c.h_group_not[g] = (4 * nm + kTileW - 1) / kTileW;
        ot += c.h_group_not[g];
    }
    c.n_occ_tiles = ot;
    int vt = ot;
    for (int g = 0; g < G; ++g) {
        c.h_group_vt0[g] = vt;
        c.h_group_nvt[g] = (2 * c.h_group_nmol[g] + kTileW - 1) / kTileW;
        vt += c.h_group_nvt[g];
    }
    c.n_tiles = vt;
    c.h_tile_group.assign(c.n_tiles, 0);
    c.h_tile_kind.assign(c.n_tiles, 0);
    c.h_tile_loc0.assign(c.n_tiles, 0);
    c.h_tile_nmo.assign(c.n_tiles, 0);
    c.h_tile_mo0.assign(c.n_tiles, 0);
    for (int g = 0; g < G; ++g) {
        int no = 4 * c.h_group_nmol[g], nv = 2 * c.h_group_nmol[g];
        for (int t = 0; t < c.h_group_not[g]; ++t) {
            int id = c.h_group_ot0[g] + t;
            c.h_tile_group[id] = g;
            c.h_tile_kind[id] = 0;
            c.h_tile_loc0[id] = t * kTileW;
            c.h_tile_nmo[id] = std::min(kTileW, no - t * kTileW);
            c.h_tile_mo0[id] = c.h_group_occ0[g] + t * kTileW;
        }
        for (int t = 0; t < c.h_group_nvt[g]; ++t) {
            int id = c.h_group_vt0[g] + t;
            c.h_tile_group[id] = g;
            c.h_tile_kind[id] = 1;
            c.h_tile_loc0[id] = t * kTileW;
            c.h_tile_nmo[id] = std::min(kTileW, nv - t * kTileW);
            c.h_tile_mo0[id] = c.h_group_virt0[g] + t * kTileW;
        }
    }

    // ---- group neighbour map: some atom pair closer than group_cut ----
    std::vector<double> gc(3 * G, 0.0), grad(G, 0.0);
    std::vector<std::vector<int>> gatoms(G);
    for (int g = 0; g < G; ++g) {
        for (int m : mols[g])
            for (int a = 0; a < 3; ++a) gatoms[g].push_back(3 * m + a);
        for (int a : gatoms[g])
            for (int d = 0; d < 3; ++d) gc[3 * g + d] += X[3 * a + d];
        for (int d = 0; d < 3; ++d) gc[3 * g + d] /= (double)gatoms[g].size();
        for (int a : gatoms[g]) grad[g] = std::max(grad[g], std::sqrt(dist2(&gc[3 * g], &X[3 * a])));
    }
    double gmax = *std::max_element(grad.begin(), grad.end());
    const double gc2 = c.prm.group_cut * c.prm.group_cut;
    // groups of a cluster are consecutive (checked above): one cell grid per cluster
    c.h_cl_g0.assign(c.n_clusters + 1, G);
    for (int g = G - 1; g >= 0; --g) c.h_cl_g0[c.h_mol_cluster[mols[g][0]]] = g;
    for (int k = c.n_clusters - 1; k >= 0; --k) c.h_cl_g0[k] = std::min(c.h_cl_g0[k], c.h_cl_g0[k + 1]);
    std::vector<std::vector<int>> gnb(G);
    for (int k = 0; k < c.n_clusters; ++k) {
        const int g0 = c.h_cl_g0[k], ng = c.h_cl_g0[k + 1] - g0;
        if (ng <= 0) continue;
        std::vector<double> gck(gc.begin() + 3 * (size_t)g0, gc.begin() + 3 * (size_t)(g0 + ng));
        CellGrid gg;
        gg.build(gck, ng, c.prm.group_cut + 2.0 * gmax + 1e-9);
        for (int A = g0; A < g0 + ng; ++A) {
            int cx = gg.coord(&gc[3 * A], 0), cy = gg.coord(&gc[3 * A], 1), cz = gg.coord(&gc[3 * A], 2);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int x = cx + dx, y = cy + dy, z = cz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= gg.n[0] || y >= gg.n[1] || z >= gg.n[2]) continue;
                        for (int Bl = gg.head[x + gg.n[0] * (y + gg.n[1] * z)]; Bl >= 0; Bl = gg.next[Bl]) {
                            const int B = g0 + Bl;
                            bool hit = (A == B);
                            for (size_t i = 0; i < gatoms[A].size() && !hit; ++i)
                                for (size_t j = 0; j < gatoms[B].size() && !hit; ++j)
                                    if (dist2(&X[3 * gatoms[A][i]], &X[3 * gatoms[B][j]]) < gc2) hit = true;
                            if (hit) gnb[A].push_back(B);
                        }
                    }
            std::sort(gnb[A].begin(), gnb[A].end());
        }
    }
    // ---- greedy first-fit edge colouring, edges {A < B} in lexicographic order ----
    std::vector<std::vector<char>> used(G);
    std::vector<std::vector<int>> ecol(G);
    int n_col = 1;
    for (int A = 0; A < G; ++A) ecol[A].assign(gnb[A].size(), -1);
    for (int A = 0; A < G; ++A) {
        for (size_t k = 0; k < gnb[A].size(); ++k) {
            int B = gnb[A][k];
            if (B == A) {
                ecol[A][k] = 0;
                continue;
            }
            if (B < A) continue;
            int col = 1;
            while ((col < (int)used[A].size() && used[A][col]) || (col < (int)used[B].size() && used[B][col])) ++col;
            ecol[A][k] = col;
            if ((int)used[A].size() <= col) used[A].resize(col + 1, 0);
            if ((int)used[B].size() <= col) used[B].resize(col + 1, 0);
            used[A][col] = used[B][col] = 1;
            n_col = std::max(n_col, col + 1);
        }
    }
    for (int A = 0; A < G; ++A)
        for (size_t k = 0; k < gnb[A].size(); ++k) {
            int B = gnb[A][k];
            if (B < A) {
                auto it = std::lower_bound(gnb[B].begin(), gnb[B].end(), A);
                ecol[A][k] = ecol[B][it - gnb[B].begin()];
            }
        }
    c.n_colours = n_col;
    c.h_gnb_ptr.assign(G + 1, 0);
    for (int A = 0; A < G; ++A) c.h_gnb_ptr[A + 1] = c.h_gnb_ptr[A] + (int)gnb[A].size();
    c.n_gnb = c.h_gnb_ptr[G];
    c.h_gnb_col.resize(c.n_gnb);
    c.h_gnb_row.resize(c.n_gnb);
    c.h_gnb_colour.resize(c.n_gnb);
    for (int A = 0; A < G; ++A)
        for (size_t k = 0; k < gnb[A].size(); ++k) {
            int e = c.h_gnb_ptr[A] + (int)k;
            c.h_gnb_col[e] = gnb[A][k];
            c.h_gnb_row[e] = A;
            c.h_gnb_colour[e] = ecol[A][k];
        }
    // blocks by colour: all directed blocks, and blocks with A <= B
    c.h_colour_ptr.assign(n_col + 1, 0);
    c.h_ocolour_ptr.assign(n_col + 1, 0);
    for (int e = 0; e < c.n_gnb; ++e) {
        c.h_colour_ptr[c.h_gnb_colour[e] + 1]++;
        if (c.h_gnb_row[e] <= c.h_gnb_col[e]) c.h_ocolour_ptr[c.h_gnb_colour[e] + 1]++;
    }
    for (int k = 0; k < n_col; ++k) {
        c.h_colour_ptr[k + 1] += c.h_colour_ptr[k];
        c.h_ocolour_ptr[k + 1] += c.h_ocolour_ptr[k];
    }
    c.h_colour_blk.assign(c.n_gnb, 0);
    c.h_ocolour_blk.assign(c.h_ocolour_ptr[n_col], 0);
    {
        std::vector<int> f1(c.h_colour_ptr.begin(), c.h_colour_ptr.end() - 1);
        std::vector<int> f2(c.h_ocolour_ptr.begin(), c.h_ocolour_ptr.end() - 1);
        for (int e = 0; e < c.n_gnb; ++e) {
            int col = c.h_gnb_colour[e];
            c.h_colour_blk[f1[col]++] = e;
            if (c.h_gnb_row[e] <= c.h_gnb_col[e]) c.h_ocolour_blk[f2[col]++] = e;
        }
        // within each colour, blocks between full groups (8 molecules: 32
        // occupied and 16 virtual MOs) first; FP32 sweeps run them through the
        // register-resident kernel (occupied passes: A != B only)
        auto full_first = [&](std::vector<int>& blk, const std::vector<int>& ptr, std::vector<int>& nfull,
                              bool distinct) {
            nfull.assign(n_col, 0);
            for (int k = 0; k < n_col; ++k) {
                auto b = blk.begin() + ptr[k], en = blk.begin() + ptr[k + 1];
                auto mid = std::stable_partition(b, en, [&](int e) {
                    const int A = c.h_gnb_row[e], B = c.h_gnb_col[e];
                    return (!distinct || A != B) && c.h_group_nmol[A] == kMaxMolPerGroup &&
                           c.h_group_nmol[B] == kMaxMolPerGroup;
                });
                nfull[k] = (int)(mid - b);
            }
        };
        full_first(c.h_colour_blk, c.h_colour_ptr, c.h_colour_nfull, false);
        full_first(c.h_ocolour_blk, c.h_ocolour_ptr, c.h_ocolour_nfull, true);
    }

    // ---- tile pairs of the occupied-virtual transform ----
    // block e = (A, B): a in occ tiles of A, b in virt tiles of B
    std::vector<std::vector<std::pair<int, int>>> by_a(c.n_tiles);
    c.h_rot_blk_tp0.assign(c.n_gnb, 0);
    int out = 0;
    for (int e = 0; e < c.n_gnb; ++e) {
        int A = c.h_gnb_row[e], B = c.h_gnb_col[e];
        c.h_rot_blk_tp0[e] = out;
        for (int ia = 0; ia < c.h_group_not[A]; ++ia)
            for (int ib = 0; ib < c.h_group_nvt[B]; ++ib)
                by_a[c.h_group_ot0[A] + ia].push_back({c.h_group_vt0[B] + ib, out++});
    }
    c.n_rot_tp = out;
    c.h_rot_tp_ptr.assign(c.n_tiles + 1, 0);
    for (int t = 0; t < c.n_tiles; ++t) c.h_rot_tp_ptr[t + 1] = c.h_rot_tp_ptr[t] + (int)by_a[t].size();
    c.h_rot_tp_b.resize(out);
    c.h_rot_tp_out.resize(out);
    for (int t = 0; t < c.n_tiles; ++t)
        for (size_t k = 0; k < by_a[t].size(); ++k) {
            c.h_rot_tp_b[c.h_rot_tp_ptr[t] + k] = by_a[t][k].first;
            c.h_rot_tp_out[c.h_rot_tp_ptr[t] + k] = by_a[t][k].second;
        }
    (void)sys;
    (void)nA;
    return SSCF_OK;
}

// Tile pairs of the overlap transform for a pass over all MOs (w = 0) or the
// occupied MOs only (w = 1): blocks (A, B) with A <= B; the side of a group
// lists its occupied tiles, then (w = 0) its virtual tiles.
void ortho_lists(const Ctx& c, int w, std::vector<int>& ptr, std::vector<int>& bl, std::vector<int>& outl,
                 std::vector<int>& blk_tp, int& n_tp) {
    std::vector<std::vector<std::pair<int, int>>> by_a(c.n_tiles);
    blk_tp.assign((size_t)c.n_gnb * 9, -1);
    int out = 0;
    auto side = [&](int g, int* t) {
        int n = 0;
        for (int i = 0; i < c.h_group_not[g]; ++i) t[n++] = c.h_group_ot0[g] + i;
        if (w == 0)
            for (int i = 0; i < c.h_group_nvt[g]; ++i) t[n++] = c.h_group_vt0[g] + i;
        return n;
    };
    for (int e = 0; e < c.n_gnb; ++e) {
        int A = c.h_gnb_row[e], B = c.h_gnb_col[e];
        if (A > B) continue;
        int ta[3], tb[3];
        int na = side(A, ta), nb = side(B, tb);
        for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j) {
                if (A == B && j < i) continue;
                blk_tp[(size_t)e * 9 + i * 3 + j] = out;
                by_a[ta[i]].push_back({tb[j], out++});
            }
    }
    n_tp = out;
    ptr.assign(c.n_tiles + 1, 0);
    for (int t = 0; t < c.n_tiles; ++t) ptr[t + 1] = ptr[t] + (int)by_a[t].size();
    bl.resize(out);
    outl.resize(out);
    for (int t = 0; t < c.n_tiles; ++t)
        for (size_t k = 0; k < by_a[t].size(); ++k) {
            bl[ptr[t] + k] = by_a[t][k].first;
            outl[ptr[t] + k] = by_a[t][k].second;
        }
}

template <typename V>
int upload(Ctx& c, V** d, const std::vector<V>& h) {
    size_t n = std::max<size_t>(h.size(), 1);
    CKS(dalloc(&c, d, n));
    if (!h.empty()) CK(cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return SSCF_OK;
}

// Records one CUDA event pair on the context's stream around a launcher when
// profiling is on; the times are summed per name at the next sscf_profile_read.
struct ProfScope {
    Ctx& c;
    int id = -1;
    cudaEvent_t e0 = nullptr;
    ProfScope(Ctx& cc, const char* name) : c(cc) {
        if (!c.prof) return;
        for (size_t i = 0; i < c.prof_names.size(); ++i)
            if (c.prof_names[i] == name) id = (int)i;
        if (id < 0) {
            id = (int)c.prof_names.size();
            c.prof_names.push_back(name);
            c.prof_ms.push_back(0.0);
            c.prof_calls.push_back(0);
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventRecord(e0, c.stream) != cudaSuccess) {
            cudaGetLastError();
            e0 = nullptr;
        }
    }
    ~ProfScope() {
        if (!c.prof || !e0) return;
        cudaEvent_t e1 = nullptr;
        if (cudaEventCreate(&e1) != cudaSuccess || cudaEventRecord(e1, c.stream) != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(e0);
            return;
        }
        c.prof_pending.push_back({id, e0, e1});
    }
};

int prof_collect(Ctx& c) {
    if (c.prof_pending.empty()) return SSCF_OK;
    CK(cudaStreamSynchronize(c.stream));
    for (auto& r : c.prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            c.prof_ms[r.id] += ms;
            c.prof_calls[r.id] += 1;
        } else {
            cudaGetLastError();
        }
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    c.prof_pending.clear();
    return SSCF_OK;
}

#define PK(name, call)            \
    do {                          \
        ProfScope ps_(c, name);   \
        CK(call);                 \
    } while (0)

// Storage-type conversion of n values (FP32 <-> FP64).
template <typename S, typename D>
__global__ void k_convert(size_t n, const S* __restrict__ in, D* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (D)in[i];
}

// Convergence test of one SCC iteration inside a graph-resident stage (the
// test of sscf_run's host loop: every cluster with max |q - q_prev| <= dq_tol
// and |E - E_prev| <= e_tol). Sets the condition of the stage's while node:
// another iteration unless all clusters converged, the iteration limit is
// reached, a kernel of the iteration set an error bit, or an energy is not
// finite. One block.
__global__ void k_scc_loop_test(int n_clusters, const double* __restrict__ cl_E, double* __restrict__ cl_Eprev,
                                const double* __restrict__ cl_dq, double dq_tol, double e_tol, int max_iter,
                                int* __restrict__ loop, const unsigned* __restrict__ err,
                                cudaGraphConditionalHandle handle) {
    __shared__ int s_ok, s_bad;
    if (threadIdx.x == 0) {
        s_ok = 1;
        s_bad = 0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_clusters; k += blockDim.x) {
        const double e = cl_E[k];
        if (!isfinite(e)) s_bad = 1;
        if (!(cl_dq[k] <= dq_tol && fabs(e - cl_Eprev[k]) <= e_tol)) s_ok = 0;
        cl_Eprev[k] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int it = loop[0] + 1;
        loop[0] = it;
        loop[1] = s_ok;
        const bool stop = s_ok || it >= max_iter || s_bad || (*err & (kErrCapacity | kErrSortSize | kErrNonFinite));
        cudaGraphSetConditional(handle, stop ? 0u : 1u);
    }
}

void drop_graph(Ctx& c) {
    if (c.graph_exec) cudaGraphExecDestroy(c.graph_exec);
    if (c.graph) cudaGraphDestroy(c.graph);
    c.graph_exec = nullptr;
    c.graph = nullptr;
    c.graph_valid = false;
}

// Target of an orthonormalisation (Section "Sparsity and numerical accuracy":
// eps / 100), floored at what the storage precision resolves: 32 u_fp32 =
// 2^-19 for FP32 storage, where eps / 100 can lie below the rounding of the
// stored MOs, and 1e-13 for FP64 storage, where it matters only as eps -> 0.
double ortho_target(const Ctx& c, double eps) {
    const double floor_ = c.prec == SSCF_MIXED ? 32.0 * 0x1p-24 : 1e-13;
    return std::max(eps / 100.0, floor_);
}

int sync_scalars(Ctx& c) {
    CK(cudaMemcpyAsync(c.h_sc, c.d_sc, sizeof(DeviceScalars), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (c.h_sc->err & kErrCapacity) return SSCF_ERR_CAPACITY;
    if (c.h_sc->err & kErrSortSize) return SSCF_ERR_CAPACITY;
    if (c.h_sc->err & kErrNonFinite) return SSCF_ERR_NONFINITE;
    if (c.h_sc->err & kErrGuess) return SSCF_ERR_NONFINITE;
    return SSCF_OK;
}

}  // namespace

namespace sscf {

int dev_alloc(Ctx* c, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    void* q = nullptr;
    if (g_alloc) {
        q = g_alloc(bytes, g_alloc_user);
        if (!q) return SSCF_ERR_OOM;
    } else {
        if (cudaMalloc(&q, bytes) != cudaSuccess) {
            cudaGetLastError();
            return SSCF_ERR_OOM;
        }
    }
    c->allocations.push_back(q);
    *p = q;
    return SSCF_OK;
}

void* raw_alloc(size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    void* q = nullptr;
    if (g_alloc) return g_alloc(bytes, g_alloc_user);
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return q;
}

void raw_free(void* p) {
    if (!p) return;
    if (g_free)
        g_free(p, g_alloc_user);
    else
        cudaFree(p);
}

void dev_release(Ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocations.size(); ++i)
        if (c->allocations[i] == p) {
            c->allocations.erase(c->allocations.begin() + (long)i);
            break;
        }
    if (g_free)
        g_free(p, g_alloc_user);
    else
        cudaFree(p);
}

void dev_free_all(Ctx* c) {
    for (void* q : c->allocations) {
        if (g_free)
            g_free(q, g_alloc_user);
        else
            cudaFree(q);
    }
    c->allocations.clear();
}

}  // namespace sscf

// ============================================================================
// C-ABI
// ============================================================================

extern "C" {

const char* sscf_strerror(int s) {
    switch (s) {
        case SSCF_OK: return "ok";
        case SSCF_ERR_INVALID_ARG: return "invalid argument";
        case SSCF_ERR_OOM: return "device allocation failed";
        case SSCF_ERR_CUDA: return "CUDA error";
        case SSCF_ERR_NONFINITE: return "non-finite value";
        case SSCF_ERR_CAPACITY: return "sparse capacity exceeded";
        case SSCF_ERR_NOT_CONVERGED: return "SCF not converged";
        case SSCF_ERR_TIMEOUT: return "device wait timed out";
        case SSCF_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

int sscf_set_allocator(sscf_alloc_fn alloc, sscf_free_fn free_, void* user) {
    if ((alloc == nullptr) != (free_ == nullptr)) return SSCF_ERR_INVALID_ARG;
    g_alloc = alloc;
    g_free = free_;
    g_alloc_user = user;
    return SSCF_OK;
}

int sscf_create(const sscf_system* sys, const sscf_params* prm, void* cuda_stream, sscf_ctx** out) {
    if (!sys || !prm || !out || !sys->species || !sys->xyz || !sys->group_of_mol) return SSCF_ERR_INVALID_ARG;
    *out = nullptr;
    if (sys->n_atoms <= 0 || sys->n_atoms % 3 != 0) return SSCF_ERR_INVALID_ARG;
    if (prm->precision != SSCF_FP64 && prm->precision != SSCF_MIXED) return SSCF_ERR_INVALID_ARG;
    if (prm->apply_variant < 0 || prm->apply_variant > 2) return SSCF_ERR_INVALID_ARG;
    if (prm->closure_mode < 0) return SSCF_ERR_INVALID_ARG;
    if (prm->cap_tiles < 0 || prm->cap_y < 0) return SSCF_ERR_INVALID_ARG;
    if (!(prm->r_cut > 0) || !(prm->r_decay > 0) || !(prm->group_cut > 0) || !(prm->eps >= 0) ||
        !(prm->U[0] > 0) || !(prm->U[1] > 0) || !(prm->rot_cap_factor > 0))
        return SSCF_ERR_INVALID_ARG;
    for (int a = 0; a < sys->n_atoms; ++a) {
        int want = (a % 3 == 0) ? 0 : 1;
        if (sys->species[a] != want) return SSCF_ERR_INVALID_ARG;
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(sys->xyz[3 * a + d])) return SSCF_ERR_NONFINITE;
    }
    sscf_ctx* h = new (std::nothrow) sscf_ctx();
    if (!h) return SSCF_ERR_OOM;
    Ctx& c = h->c;
    c.prm = *prm;
    c.stream = (cudaStream_t)cuda_stream;
    c.prec = prm->precision;
    c.tsize = c.prec == SSCF_FP64 ? 8 : 4;
    c.n_atoms = sys->n_atoms;
    c.n_mol = sys->n_atoms / 3;
    c.n_ao = 6 * c.n_mol;
    c.n_occ = 4 * c.n_mol;
    c.n_mo = 6 * c.n_mol;
    c.h_species.assign(sys->species, sys->species + c.n_atoms);
    c.h_xyz.assign(sys->xyz, sys->xyz + 3 * c.n_atoms);
    c.h_mol_group.assign(sys->group_of_mol, sys->group_of_mol + c.n_mol);
    c.h_mol_cluster.assign(c.n_mol, 0);
    if (sys->cluster_of_mol) c.h_mol_cluster.assign(sys->cluster_of_mol, sys->cluster_of_mol + c.n_mol);
    c.n_clusters = 0;
    for (int m = 0; m < c.n_mol; ++m) {
        const int cl = c.h_mol_cluster[m];
        const int prev = m ? c.h_mol_cluster[m - 1] : -1;
        if (cl != prev && cl != prev + 1) {   // clusters consecutive and numbered in order
            delete h;
            return SSCF_ERR_INVALID_ARG;
        }
        c.n_clusters = cl + 1;
    }
    c.h_cl_mol0.assign(c.n_clusters, 0);
    c.h_cl_nmol.assign(c.n_clusters, 0);
    for (int m = c.n_mol - 1; m >= 0; --m) {
        c.h_cl_mol0[c.h_mol_cluster[m]] = m;
        c.h_cl_nmol[c.h_mol_cluster[m]]++;
    }
    int G = 0;
    for (int m = 0; m < c.n_mol; ++m) {
        if (c.h_mol_group[m] < 0) {
            delete h;
            return SSCF_ERR_INVALID_ARG;
        }
        G = std::max(G, c.h_mol_group[m] + 1);
    }
    c.n_groups = G;
    int st = build_structure(c, sys);
    if (st != SSCF_OK) {
        delete h;
        return st;
    }
    auto fail = [&](int s) {
        dev_free_all(&c);
        if (c.h_sc) cudaFreeHost(c.h_sc);
        delete h;
        return s;
    };
    // per-cluster sizes: a row of C only holds tiles of its own cluster, a
    // column of Y only rows of its own cluster
    {
        std::vector<int> cl_tiles(c.n_clusters, 0), cl_otiles(c.n_clusters, 0);
        std::vector<int> g_cl(c.n_groups, 0);
        for (int m = 0; m < c.n_mol; ++m) g_cl[c.h_mol_group[m]] = c.h_mol_cluster[m];
        for (int t = 0; t < c.n_tiles; ++t) {
            cl_tiles[g_cl[c.h_tile_group[t]]]++;
            if (c.h_tile_kind[t] == 0) cl_otiles[g_cl[c.h_tile_group[t]]]++;
        }
        c.max_cl_tiles = *std::max_element(cl_tiles.begin(), cl_tiles.end());
        c.max_cl_otiles = *std::max_element(cl_otiles.begin(), cl_otiles.end());
        c.max_cl_mol = *std::max_element(c.h_cl_nmol.begin(), c.h_cl_nmol.end());
    }
    c.cap = prm->cap_tiles > 0 ? std::min(prm->cap_tiles, c.max_cl_tiles) : c.max_cl_tiles;
    c.cap = std::max(c.cap, 2);
    c.max_cl_groups = 0;
    for (int k = 0; k < c.n_clusters; ++k) c.max_cl_groups = std::max(c.max_cl_groups, c.h_cl_g0[k + 1] - c.h_cl_g0[k]);
    // the closure keeps a row's tile list and 16-bit slots in shared memory, and
    // labels every unit of a cluster in one CTA
    if (c.cap > 32767 || closure_smem_bytes(&c) > (size_t)kMaxDynSmem ||
        closure_labels_smem_bytes(&c) > (size_t)kMaxDynSmem) {
        delete h;
        return SSCF_ERR_INVALID_ARG;
    }
    c.capY = prm->cap_y > 0 ? std::min(prm->cap_y, c.max_cl_mol) : c.max_cl_mol;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            c.n_sm = nsm;
    }
    c.apply_variant = prm->apply_variant;
    c.closure_window = prm->closure_mode;
    // uploads
#define UP(d, v)                        \
    do {                                \
        int s_ = upload(c, &d, v);      \
        if (s_ != SSCF_OK) return fail(s_); \
    } while (0)
    UP(c.d_xyz, c.h_xyz);
    UP(c.d_species, c.h_species);
    UP(c.d_mp_ptr, c.h_mp_ptr);
    UP(c.d_mp_col, c.h_mp_col);
    {
        std::vector<int> row(c.n_mp);
        for (int m = 0; m < c.n_mol; ++m)
            for (int k = c.h_mp_ptr[m]; k < c.h_mp_ptr[m + 1]; ++k) row[k] = m;
        UP(c.d_mp_row, row);
        std::vector<int> rev(c.n_mp);
        for (int m = 0; m < c.n_mol; ++m)
            for (int k = c.h_mp_ptr[m]; k < c.h_mp_ptr[m + 1]; ++k) {
                const int n = c.h_mp_col[k];
                const auto b = c.h_mp_col.begin();
                rev[k] = (int)(std::lower_bound(b + c.h_mp_ptr[n], b + c.h_mp_ptr[n + 1], m) - b);
                // the pattern is symmetric (a distance test on both orders of the pair)
                if (rev[k] >= c.h_mp_ptr[n + 1] || c.h_mp_col[rev[k]] != m) return fail(SSCF_ERR_INVALID_ARG);
            }
        UP(c.d_mp_rev, rev);
    }
    UP(c.d_mol_group, c.h_mol_group);
    UP(c.d_mol_local, c.h_mol_local);
    UP(c.d_group_nmol, c.h_group_nmol);
    UP(c.d_group_ot0, c.h_group_ot0);
    UP(c.d_group_not, c.h_group_not);
    UP(c.d_group_vt0, c.h_group_vt0);
    UP(c.d_group_nvt, c.h_group_nvt);
    UP(c.d_group_occ0_mo, c.h_group_occ0);
    UP(c.d_group_virt0_mo, c.h_group_virt0);
    c.h_self_blk.assign(c.n_groups, -1);
    for (int e = 0; e < c.n_gnb; ++e)
        if (c.h_gnb_row[e] == c.h_gnb_col[e]) c.h_self_blk[c.h_gnb_row[e]] = e;
    UP(c.d_self_blk, c.h_self_blk);
    UP(c.d_tile_group, c.h_tile_group);
    {
        std::vector<int> g_row0(c.n_groups, 0), tile_row0(c.n_tiles), mol_row0(c.n_mol), mol_ot0(c.n_mol);
        std::vector<int> cl_ot0(c.n_clusters, 1 << 30), lo(c.n_atoms), hi(c.n_atoms);
        for (int m = c.n_mol - 1; m >= 0; --m) g_row0[c.h_mol_group[m]] = c.h_cl_mol0[c.h_mol_cluster[m]];
        for (int t = 0; t < c.n_tiles; ++t) tile_row0[t] = g_row0[c.h_tile_group[t]];
        for (int m = 0; m < c.n_mol; ++m) {
            mol_row0[m] = c.h_cl_mol0[c.h_mol_cluster[m]];
            const int cl = c.h_mol_cluster[m];
            cl_ot0[cl] = std::min(cl_ot0[cl], c.h_group_ot0[c.h_mol_group[m]]);
        }
        for (int m = 0; m < c.n_mol; ++m) mol_ot0[m] = cl_ot0[c.h_mol_cluster[m]];
        for (int a2 = 0; a2 < c.n_atoms; ++a2) {
            const int cl = c.h_mol_cluster[a2 / 3];
            lo[a2] = 3 * c.h_cl_mol0[cl];
            hi[a2] = 3 * (c.h_cl_mol0[cl] + c.h_cl_nmol[cl]);
        }
        std::vector<int> group_cl(c.n_groups, 0);
        for (int m = 0; m < c.n_mol; ++m) group_cl[c.h_mol_group[m]] = c.h_mol_cluster[m];
        UP(c.d_group_cl, group_cl);
        c.h_cl_sel_init.assign((size_t)c.n_clusters * 6, 0ull);
        for (int cl = 0; cl < c.n_clusters; ++cl)
            c.h_cl_sel_init[(size_t)cl * 6 + 5] =
                (unsigned long long)(c.prm.rot_cap_factor * (double)(4 * c.h_cl_nmol[cl]));
        UP(c.d_cl_sel_init, c.h_cl_sel_init);
        UP(c.d_tile_row0, tile_row0);
        UP(c.d_mol_row0, mol_row0);
        UP(c.d_mol_ot0, mol_ot0);
        UP(c.d_mol_cluster, c.h_mol_cluster);
        UP(c.d_cl_g0, c.h_cl_g0);
        std::vector<int> cot(c.n_clusters + 1), cvt(c.n_clusters + 1);
        for (int k = 0; k <= c.n_clusters; ++k) {
            const int g = c.h_cl_g0[k];
            cot[k] = g < c.n_groups ? c.h_group_ot0[g] : c.n_occ_tiles;
            cvt[k] = g < c.n_groups ? c.h_group_vt0[g] : c.n_tiles;
        }
        UP(c.d_cl_ot0, cot);
        UP(c.d_cl_vt0, cvt);
        // blocks by cluster: gnb entries run over A, and groups over clusters, so
        // the blocks of a cluster are consecutive in both lists
        for (int w = 0; w < 2; ++w) {
            std::vector<int> ptr(c.n_clusters + 1, 0), blk;
            for (int k = 0; k < c.n_clusters; ++k) {
                for (int e = c.h_gnb_ptr[c.h_cl_g0[k]]; e < c.h_gnb_ptr[c.h_cl_g0[k + 1]]; ++e)
                    if (w == 0 || c.h_gnb_row[e] <= c.h_gnb_col[e]) blk.push_back(e);
                ptr[k + 1] = (int)blk.size();
            }
            UP(c.d_clblk_ptr[w], ptr);
            UP(c.d_clblk[w], blk);
        }
        UP(c.d_atom_lo, lo);
        UP(c.d_atom_hi, hi);
        UP(c.d_cl_mol0, c.h_cl_mol0);
        UP(c.d_cl_nmol, c.h_cl_nmol);
    }
    UP(c.d_tile_kind, c.h_tile_kind);
    UP(c.d_tile_loc0, c.h_tile_loc0);
    UP(c.d_tile_nmo, c.h_tile_nmo);
    UP(c.d_tile_mo0, c.h_tile_mo0);
    UP(c.d_gnb_ptr, c.h_gnb_ptr);
    UP(c.d_gnb_row, c.h_gnb_row);
    UP(c.d_gnb_col, c.h_gnb_col);
    UP(c.d_gnb_colour, c.h_gnb_colour);
    UP(c.d_colour_ptr, c.h_colour_ptr);
    UP(c.d_colour_blk, c.h_colour_blk);
    UP(c.d_ocolour_ptr, c.h_ocolour_ptr);
    UP(c.d_ocolour_blk, c.h_ocolour_blk);
    UP(c.d_rot_tp_ptr, c.h_rot_tp_ptr);
    UP(c.d_rot_tp_b, c.h_rot_tp_b);
    UP(c.d_rot_tp_out, c.h_rot_tp_out);
    UP(c.d_rot_blk_tp0, c.h_rot_blk_tp0);
    {
        std::vector<int> dp(c.n_tiles + 1), db(c.n_tiles), dout(c.n_tiles);
        for (int t = 0; t <= c.n_tiles; ++t) dp[t] = t;
        for (int t = 0; t < c.n_tiles; ++t) db[t] = dout[t] = t;
        UP(c.d_diag_tp_ptr, dp);
        UP(c.d_diag_tp_b, db);
        UP(c.d_diag_tp_out, dout);
    }
    int max_ort = 0;
    for (int w = 0; w < 2; ++w) {
        std::vector<int> p, b, o;
        ortho_lists(c, w, p, b, o, c.h_ort_blk_tp[w], c.n_ort_tp[w]);
        UP(c.d_ort_tp_ptr[w], p);
        UP(c.d_ort_tp_b[w], b);
        UP(c.d_ort_tp_out[w], o);
        UP(c.d_ort_blk_tp[w], c.h_ort_blk_tp[w]);
        max_ort = std::max(max_ort, c.n_ort_tp[w]);
    }
#undef UP
    const size_t ts = c.tsize;
#define AL(p, n)                                    \
    do {                                            \
        int s_ = dev_alloc(&c, (void**)&(p), (n));  \
        if (s_ != SSCF_OK) return fail(s_);         \
    } while (0)
    AL(c.d_H0b, (size_t)c.n_mp * 36 * 8);
    AL(c.d_Sb, (size_t)c.n_mp * 36 * 8);
    AL(c.d_dens_part, (size_t)c.n_mp * 4 * 8);
    AL(c.d_Hb, (size_t)c.n_mp * 36 * ts);
    AL(c.d_Sbt, (size_t)c.n_mp * 36 * ts);
    for (int b = 0; b < 2; ++b) {
        AL(c.d_c_nt[b], (size_t)c.n_mol * 4);
        AL(c.d_c_tile[b], (size_t)c.n_mol * c.cap * 4);
        AL(c.d_c_val[b], (size_t)c.n_mol * c.cap * kTileVals * ts);
        AL(c.d_c_nz[b], (size_t)c.n_mol * c.cap);
        if (b == 0) {
            AL(c.d_unit_lab, (size_t)2 * c.n_groups * 4);
            AL(c.d_lab_start, (size_t)2 * c.n_groups * 4);
            AL(c.d_lab_cnt, (size_t)2 * c.n_groups * 4);
            AL(c.d_lab_mem, (size_t)2 * c.n_groups * 4);
        }
    }
    AL(c.d_cci_ptr, (size_t)(c.n_tiles + 1) * 4);
    AL(c.d_cci_cnt, (size_t)c.n_tiles * 4);
    AL(c.d_cci_row, (size_t)c.n_mol * c.cap * 4);
    AL(c.d_cci_slot, (size_t)c.n_mol * c.cap * 4);
    AL(c.d_c_cnz, (size_t)c.n_mol * c.cap);
    AL(c.d_blk_info, (size_t)std::max(c.n_gnb, 1) * 8 * 4);
    AL(c.d_y_n, (size_t)c.n_tiles * 4);
    AL(c.d_y_row, (size_t)c.n_tiles * c.capY * 4);
    AL(c.d_y_val, (size_t)c.n_tiles * c.capY * kTileVals * ts);
    AL(c.d_F, (size_t)std::max(c.n_rot_tp, 1) * 256 * ts);
    AL(c.d_Fdiag_tiles, (size_t)c.n_tiles * 256 * ts);
    AL(c.d_Fd, (size_t)c.n_mo * 8);
    AL(c.d_sig, (size_t)std::max(max_ort, 1) * 256 * ts);
    AL(c.d_scale, (size_t)c.n_mo * 8);
    AL(c.d_pr_n, (size_t)c.n_gnb * 4);
    AL(c.d_pr_lvl, (size_t)c.n_gnb * (kMaxSub + 1) * 4);
    AL(c.d_pr_ij, (size_t)c.n_gnb * kOrthoCap * 2);
    AL(c.d_pr_cs, (size_t)c.n_gnb * kOrthoCap * 2 * ts);
    AL(c.d_pr_touch, (size_t)c.n_gnb * 4);
    AL(c.d_q, (size_t)c.n_atoms * 8);
    AL(c.d_q_prev, (size_t)c.n_atoms * 8);
    AL(c.d_dq_in, (size_t)c.n_atoms * 8);
    AL(c.d_Q_in, (size_t)c.n_atoms * 8);
    AL(c.d_dq, (size_t)c.n_atoms * 8);
    AL(c.d_Q, (size_t)c.n_atoms * 8);
    AL(c.d_e_mol, (size_t)c.n_mol * 8);
    AL(c.d_red, (size_t)(c.n_mol + 4096) * 8);
    AL(c.d_cl_E, (size_t)c.n_clusters * 8);
    AL(c.d_cl_sel, (size_t)c.n_clusters * 6 * 8);
    AL(c.d_cl_hist, (size_t)c.n_clusters * 256 * 8);
    AL(c.d_cl_eta, (size_t)c.n_clusters * 8);
    AL(c.d_cl_dq, (size_t)c.n_clusters * 8);
    AL(c.d_cl_Eprev, (size_t)c.n_clusters * 8);
    AL(c.d_loop, 16);
    AL(c.d_grad, (size_t)c.n_atoms * 3 * 8);
    AL(c.d_par, 8 * 8);
    AL(c.d_gmol, (size_t)c.n_mol * 9 * 8);
    AL(c.d_pmol, (size_t)c.n_mol * 8 * 8);
    AL(c.d_sc, sizeof(DeviceScalars));
#undef AL
    if (cudaMallocHost((void**)&c.h_sc, sizeof(DeviceScalars)) != cudaSuccess) {
        cudaGetLastError();
        c.h_sc = nullptr;
        return fail(SSCF_ERR_OOM);
    }
    if (cudaMemsetAsync(c.d_sc, 0, sizeof(DeviceScalars), c.stream) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (cudaMemsetAsync(c.d_cl_hist, 0, (size_t)c.n_clusters * 256 * 8, c.stream) != cudaSuccess)
        return fail(SSCF_ERR_CUDA);
    for (double* p : {c.d_q, c.d_q_prev, c.d_dq_in, c.d_Q_in, c.d_dq, c.d_Q})
        if (cudaMemsetAsync(p, 0, (size_t)c.n_atoms * 8, c.stream) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    for (int b = 0; b < 2; ++b)
        if (cudaMemsetAsync(c.d_c_nt[b], 0, (size_t)c.n_mol * 4, c.stream) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (launch_sk_blocks(&c) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (launch_build_h(&c, c.prm.eps) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    *out = h;
    return SSCF_OK;
}

void sscf_destroy(sscf_ctx* h) {
    if (!h) return;
    cudaStreamSynchronize(h->c.stream);
    prof_collect(h->c);
    drop_graph(h->c);
    dev_free_all(&h->c);
    if (h->c.h_sc) cudaFreeHost(h->c.h_sc);
    delete h;
}

int sscf_set_thresholds(sscf_ctx* h, double eps, double dq_tol, double e_tol) {
    if (!h || !(eps >= 0) || !(dq_tol >= 0) || !(e_tol >= 0)) return SSCF_ERR_INVALID_ARG;
    if (h->c.prm.eps != eps) drop_graph(h->c);
    h->c.prm.eps = eps;
    h->c.prm.dq_tol = dq_tol;
    h->c.prm.e_tol = e_tol;
    return SSCF_OK;
}

int sscf_set_precision(sscf_ctx* h, int precision) {
    if (!h || (precision != SSCF_FP64 && precision != SSCF_MIXED)) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (precision == c.prec) return SSCF_OK;
    drop_graph(c);
    CK(cudaStreamSynchronize(c.stream));
    const size_t ts = precision == SSCF_FP64 ? 8 : 4;
    int max_ort = std::max(std::max(c.n_ort_tp[0], c.n_ort_tp[1]), 1);
    // every buffer whose element type follows the storage precision, with its value count
    void** bufs[] = {&c.d_Hb, &c.d_Sbt, &c.d_c_val[0], &c.d_c_val[1], &c.d_y_val,
                     &c.d_F, &c.d_Fdiag_tiles, &c.d_sig, &c.d_pr_cs};
    const size_t counts[] = {(size_t)c.n_mp * 36, (size_t)c.n_mp * 36, (size_t)c.n_mol * c.cap * kTileVals,
                             (size_t)c.n_mol * c.cap * kTileVals, (size_t)c.n_tiles * c.capY * kTileVals,
                             (size_t)std::max(c.n_rot_tp, 1) * 256, (size_t)c.n_tiles * 256, (size_t)max_ort * 256,
                             (size_t)c.n_gnb * kOrthoCap * 2};
    constexpr int nb = sizeof(counts) / sizeof(counts[0]);
    void* fresh[nb] = {nullptr};
    for (int i = 0; i < nb; ++i) {
        if (dev_alloc(&c, &fresh[i], counts[i] * ts) != SSCF_OK) {
            for (int j = 0; j < i; ++j) dev_release(&c, fresh[j]);
            return SSCF_ERR_OOM;   // the context is unchanged
        }
    }
    // only the current C buffer holds state; H and S in storage precision are
    // rebuilt below, everything else is rewritten by the next step
    const int cb = 2 + c.cur;
    const size_t n = counts[cb];
    const int th = 256, blocks = (int)std::min<size_t>((n + th - 1) / th, (size_t)c.n_sm * 16);
    if (precision == SSCF_FP64)
        k_convert<float, double><<<blocks, th, 0, c.stream>>>(n, (const float*)*bufs[cb], (double*)fresh[cb]);
    else
        k_convert<double, float><<<blocks, th, 0, c.stream>>>(n, (const double*)*bufs[cb], (float*)fresh[cb]);
    c.n_launch += 1;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c.stream) != cudaSuccess) {
        cudaGetLastError();
        for (int j = 0; j < nb; ++j) dev_release(&c, fresh[j]);
        return SSCF_ERR_CUDA;
    }
    for (int i = 0; i < nb; ++i) {
        dev_release(&c, *bufs[i]);
        *bufs[i] = fresh[i];
    }
    c.prec = precision;
    c.prm.precision = precision;
    c.tsize = ts;
    CK(launch_build_h(&c, c.prm.eps));
    CK(cudaStreamSynchronize(c.stream));
    return SSCF_OK;
}

int sscf_get_dims(const sscf_ctx* h, int* n_ao, int* n_mo, int* n_occ, int* n_groups, int* n_tiles,
                  int* n_colours) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    const Ctx& c = h->c;
    if (n_ao) *n_ao = c.n_ao;
    if (n_mo) *n_mo = c.n_mo;
    if (n_occ) *n_occ = c.n_occ;
    if (n_groups) *n_groups = c.n_groups;
    if (n_tiles) *n_tiles = c.n_tiles;
    if (n_colours) *n_colours = c.n_colours;
    return SSCF_OK;
}

int sscf_guess(sscf_ctx* h) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    CK(cudaMemsetAsync(c.d_sc, 0, sizeof(unsigned), c.stream));
    CK(launch_guess(&c));
    CKS(sync_scalars(c));
    c.have_guess = true;
    c.have_e_prev = false;
    c.iteration = 0;
    return SSCF_OK;
}

int sscf_build_fock(sscf_ctx* h) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    PK("build_fock", launch_build_h(&c, c.prm.eps));
    return SSCF_OK;
}

int sscf_set_fock_blocks(sscf_ctx* h, const double* X) {
    if (!h || !X) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const size_t n = (size_t)c.n_mp * 36;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(X[i])) return SSCF_ERR_NONFINITE;
    // the same threshold as the DFTB build: off-diagonal |X_mn| < eps -> 0
    std::vector<double> v(X, X + n);
    for (int m = 0; m < c.n_mol; ++m)
        for (int e = c.h_mp_ptr[m]; e < c.h_mp_ptr[m + 1]; ++e)
            for (int u = 0; u < 36; ++u) {
                const bool diag = c.h_mp_col[e] == m && u / 6 == u % 6;
                double& x = v[(size_t)e * 36 + u];
                if (!diag && std::fabs(x) < c.prm.eps) x = 0.0;
            }
    drop_graph(c);
    CK(cudaStreamSynchronize(c.stream));
    if (c.prec == SSCF_FP64) {
        CK(cudaMemcpy(c.d_Hb, v.data(), n * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        CK(cudaMemcpy(c.d_Hb, f.data(), n * 4, cudaMemcpyHostToDevice));
    }
    return SSCF_OK;
}

int sscf_get_density_blocks(sscf_ctx* h, double* P) {
    if (!h || !P) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    if (!c.d_P) CKS(dalloc(&c, &c.d_P, (size_t)c.n_mp * 36));
    PK("density", launch_density(&c, c.d_P));
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaMemcpy(P, c.d_P, (size_t)c.n_mp * 36 * 8, cudaMemcpyDeviceToHost));
    return SSCF_OK;
}

static int rotate_sweep_async(Ctx& c) {
    PK("colindex", launch_colindex(&c));
    PK("xc_h", launch_xc_rot(&c));
    PK("transform_ov", launch_transform_rot(&c));
    PK("select_rot", launch_select_rot(&c));
    if (c.closure_window > 0) {
        for (int col = 0; col < c.n_colours; col += c.closure_window) {
            const int hi = std::min(col + c.closure_window, c.n_colours);
            PK("closure", launch_closure(&c, 0, 0, col, hi, col == 0));
            PK("colindex", launch_colindex(&c));
            PK("apply_rot", launch_apply(&c, 0, 0, col, hi));
        }
    } else {
        PK("closure", launch_closure(&c, 0, 0));
        PK("colindex", launch_colindex(&c));
        PK("apply_rot", launch_apply(&c, 0, 0));
    }
    PK("compact", launch_compact(&c));
    c.last_sched_kind = 1;
    return SSCF_OK;
}

int sscf_rotate_sweep(sscf_ctx* h, int64_t* n_rot_out, double* max_fov_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    CK(cudaMemsetAsync(c.d_sc, 0, offsetof(DeviceScalars, eta), c.stream));
    CKS(rotate_sweep_async(c));
    CKS(sync_scalars(c));
    if (n_rot_out) *n_rot_out = (int64_t)c.h_sc->n_rot;
    if (max_fov_out) *max_fov_out = c.h_sc->max_fov;
    return SSCF_OK;
}

int sscf_autotune(sscf_ctx* h, int* tf_split_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    drop_graph(c);
    // inputs of the occupied-virtual transform for the current state
    CK(launch_build_h(&c, c.prm.eps));
    CK(launch_colindex(&c));
    CK(launch_xc_rot(&c));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int cand[] = {1, 2, 4, 8};
    int best = c.tf_split, best_regs = c.tf_regs;
    float best_ms = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int regs = 0; regs < 2 && err == cudaSuccess; ++regs)
        for (int s : cand) {
            c.tf_split = s;
            c.tf_regs = regs;
            err = launch_transform_rot(&c);   // warm-up
            if (err != cudaSuccess) break;
            err = cudaEventRecord(e0, c.stream);
            for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch_transform_rot(&c);
            if (err == cudaSuccess) err = cudaEventRecord(e1, c.stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = s;
                best_regs = regs;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.tf_split = best;
    c.tf_regs = best_regs;
    if (err != cudaSuccess) return SSCF_ERR_CUDA;
    if (tf_split_out) *tf_split_out = best + 16 * best_regs;
    return SSCF_OK;
}

static int ortho_pass_async(Ctx& c, int which, double tol) {
    const int w = which == SSCF_ORTHO_OCC ? 1 : 0;
    c.ortho_tol = tol;
    PK("colindex", launch_colindex(&c));
    PK("xc_s", launch_xc(&c, false, 0, w == 1 ? c.n_occ_tiles : c.n_tiles));
    PK("transform_ss", launch_transform_ortho(&c, w));
    PK("ortho_prepare", launch_ortho_prepare(&c, w, tol));
    if (c.closure_window > 0) {
        for (int col = 0; col < c.n_colours; col += c.closure_window) {
            const int hi = std::min(col + c.closure_window, c.n_colours);
            PK("closure", launch_closure(&c, 1, w, col, hi, col == 0));
            PK("colindex", launch_colindex(&c));
            PK("apply_ortho", launch_apply(&c, 1, w, col, hi));
        }
    } else {
        PK("closure", launch_closure(&c, 1, w));
        PK("colindex", launch_colindex(&c));
        PK("apply_ortho", launch_apply(&c, 1, w));
    }
    PK("compact", launch_compact(&c));
    c.last_sched_kind = 2;
    c.last_ortho_which = w;
    return SSCF_OK;
}

int sscf_orthonormalise(sscf_ctx* h, int which, int max_pass, int* passes_out, double* eta_out) {
    if (!h || (which != SSCF_ORTHO_ALL && which != SSCF_ORTHO_OCC) || max_pass < 1) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    const double tol = ortho_target(c, c.prm.eps);
    int k = 0;
    double eta = 0.0;
    for (k = 1; k <= max_pass; ++k) {
        CK(cudaMemsetAsync(c.d_sc, 0, offsetof(DeviceScalars, e_band), c.stream));
        CKS(ortho_pass_async(c, which, tol));
        CKS(sync_scalars(c));
        eta = c.h_sc->eta;
        if (eta < tol) break;
    }
    if (k > max_pass) k = max_pass;
    if (passes_out) *passes_out = k;
    if (eta_out) *eta_out = eta;
    return SSCF_OK;
}

static int density_async(Ctx& c, bool mix) {
    PK("density", launch_density(&c));
    PK("charges_gamma", launch_charges_finish(&c, mix));
    return SSCF_OK;
}

static int finish_charges(Ctx& c, double* q_out, double* E_out, double* dq_max_out) {
    CKS(sync_scalars(c));
    if (q_out) {
        CK(cudaMemcpy(q_out, c.d_q_prev, (size_t)c.n_atoms * 8, cudaMemcpyDeviceToHost));
    }
    if (!std::isfinite(c.h_sc->energy)) return SSCF_ERR_NONFINITE;
    if (E_out) *E_out = c.h_sc->energy;
    if (dq_max_out) *dq_max_out = c.h_sc->dq_max;
    return SSCF_OK;
}

int sscf_density(sscf_ctx* h, double* q_out, double* E_out, double* dq_max_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    CK(cudaMemsetAsync(c.d_sc, 0, sizeof(unsigned), c.stream));
    CKS(density_async(c, true));
    CKS(finish_charges(c, q_out, E_out, dq_max_out));
    c.e_prev = c.h_sc->energy;
    c.have_e_prev = true;
    return SSCF_OK;
}

int sscf_reset_charges(sscf_ctx* h, double* E_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    CK(cudaMemsetAsync(c.d_sc, 0, sizeof(unsigned), c.stream));
    CKS(density_async(c, false));
    CKS(finish_charges(c, nullptr, E_out, nullptr));
    c.e_prev = c.h_sc->energy;
    c.have_e_prev = true;
    return SSCF_OK;
}

// Device part of one SCC iteration (no host synchronisation: capturable).
static int step_device(Ctx& c) {
    CK(cudaMemsetAsync(c.d_sc, 0, offsetof(DeviceScalars, hist), c.stream));
    PK("build_fock", launch_build_h(&c, c.prm.eps));
    CKS(rotate_sweep_async(c));
    if (c.prm.ortho_every) CKS(ortho_pass_async(c, SSCF_ORTHO_OCC, ortho_target(c, c.prm.eps)));
    CKS(density_async(c, true));
    CK(launch_count_tiles(&c, c.d_sc->tiles));
    return SSCF_OK;
}

// Captures step_device into a CUDA graph (once per threshold set and buffer
// parity) and replays it: one launch per SCC iteration.
static int step_graph(Ctx& c) {
    if (c.graph_valid && c.graph_cur != c.cur) drop_graph(c);
    if (!c.graph_valid) {
        const bool prof = c.prof;
        c.prof = false;
        const long long l0 = c.n_launch;
        const int cur0 = c.cur;
        CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        const int st = step_device(c);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(c.stream, &g);
        c.prof = prof;
        if (st != SSCF_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st != SSCF_OK ? st : SSCF_ERR_CUDA;
        }
        c.graph = g;
        CK(cudaGraphInstantiate(&c.graph_exec, c.graph, 0));
        c.graph_launches = c.n_launch - l0;
        c.n_launch = l0;
        c.graph_cur = cur0;
        c.graph_valid = true;
    }
    CK(cudaGraphLaunch(c.graph_exec, c.stream));
    c.n_launch += c.graph_launches;
    return SSCF_OK;
}

int sscf_enable_graph(sscf_ctx* h, int enable) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (enable && c.stream == nullptr) return SSCF_ERR_INVALID_ARG;   // the legacy stream cannot be captured
    drop_graph(c);
    c.use_graph = enable != 0;
    return SSCF_OK;
}

int sscf_step(sscf_ctx* h, sscf_step_info* info) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    const long long l0 = c.n_launch;
    if (c.use_graph)
        CKS(step_graph(c));
    else
        CKS(step_device(c));
    CKS(sync_scalars(c));
    c.iteration++;
    if (info) {
        info->energy = c.h_sc->energy;
        info->dq_max = c.h_sc->dq_max;
        info->dE = c.have_e_prev ? c.h_sc->energy - c.e_prev : c.h_sc->energy;
        info->max_fov = c.h_sc->max_fov;
        info->eta = c.h_sc->eta;
        info->n_rot = (int64_t)c.h_sc->n_rot;
        info->n_combo = (int64_t)c.h_sc->n_combo;
        info->nnz_c = (int64_t)c.h_sc->tiles[0] * kTileVals;
        info->nnz_occ = (int64_t)c.h_sc->tiles[1] * kTileVals;
        info->launches = (int64_t)(c.n_launch - l0);
        info->upd_rot = (int64_t)c.h_sc->upd[0];
        info->upd_combo = (int64_t)c.h_sc->upd[1];
        info->iteration = c.iteration;
    }
    if (!std::isfinite(c.h_sc->energy)) return SSCF_ERR_NONFINITE;
    c.e_prev = c.h_sc->energy;
    c.have_e_prev = true;
    return SSCF_OK;
}

int sscf_gradients(sscf_ctx* h, double* dE_dxyz, double* dE_dparams) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!c.have_guess) return SSCF_ERR_STATE;
    CK(cudaMemsetAsync(c.d_sc, 0, offsetof(DeviceScalars, hist), c.stream));
    // charges of the current MOs (they become the SCC input), H without threshold
    CKS(density_async(c, false));
    PK("build_fock", launch_build_h(&c, 0.0));
    // F_oo on the occupied blocks of neighbouring groups
    PK("colindex", launch_colindex(&c));
    PK("xc_h", launch_xc(&c, true, 0, c.n_occ_tiles));
    PK("transform_oo", launch_transform_ortho(&c, 1));
    PK("adjoint", launch_adjoint(&c, c.d_grad, c.d_par, c.d_gmol, c.d_pmol));
    CKS(sync_scalars(c));
    if (dE_dxyz) CK(cudaMemcpy(dE_dxyz, c.d_grad, (size_t)c.n_atoms * 3 * 8, cudaMemcpyDeviceToHost));
    if (dE_dparams) CK(cudaMemcpy(dE_dparams, c.d_par, 8 * 8, cudaMemcpyDeviceToHost));
    // restore H with the SCF threshold for later steps
    PK("build_fock", launch_build_h(&c, c.prm.eps));
    return SSCF_OK;
}

int sscf_get_cluster_results(sscf_ctx* h, double* energy, double* dq_max, int* n_clusters_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    CK(cudaStreamSynchronize(c.stream));
    if (energy) CK(cudaMemcpy(energy, c.d_cl_E, (size_t)c.n_clusters * 8, cudaMemcpyDeviceToHost));
    if (dq_max) CK(cudaMemcpy(dq_max, c.d_cl_dq, (size_t)c.n_clusters * 8, cudaMemcpyDeviceToHost));
    if (n_clusters_out) *n_clusters_out = c.n_clusters;
    return SSCF_OK;
}

int sscf_profile(sscf_ctx* h, int enable) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    CKS(prof_collect(c));
    c.prof = enable != 0;
    return SSCF_OK;
}

int sscf_profile_read(sscf_ctx* h, int max_entries, char* names, double* ms, int64_t* calls, int* n_out) {
    if (!h || max_entries < 0) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    CKS(prof_collect(c));
    const int n = (int)c.prof_names.size();
    for (int i = 0; i < n && i < max_entries; ++i) {
        if (names) {
            std::memset(names + 32 * i, 0, 32);
            std::strncpy(names + 32 * i, c.prof_names[i].c_str(), 31);
        }
        if (ms) ms[i] = c.prof_ms[i];
        if (calls) calls[i] = c.prof_calls[i];
    }
    if (n_out) *n_out = n;
    for (int i = 0; i < n; ++i) {
        c.prof_ms[i] = 0.0;
        c.prof_calls[i] = 0;
    }
    return SSCF_OK;
}

// One SCC stage as a single graph launch: an init part (iteration counter,
// previous energies) and a while node whose body is one SCC iteration
// (step_device, captured) followed by k_scc_loop_test. No host round trip
// between iterations. Returns STATE, with nothing launched, when the captured
// iteration does not end in the C buffer it starts from (it could not repeat).
static int stage_in_graph(Ctx& c, double dq_tol, double e_tol, int max_iter, bool* converged,
                          sscf_step_info* last) {
    if (!c.stream) return SSCF_ERR_STATE;
    drop_graph(c);
    const bool prof = c.prof;
    c.prof = false;
    const int cur0 = c.cur;
    const long long l0 = c.n_launch;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle;
    int st = SSCF_OK;
    long long body_launches = 0;
    auto fail = [&](int s_) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        c.prof = prof;
        c.cur = cur0;
        c.n_launch = l0;
        return s_;
    };
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return fail(SSCF_ERR_CUDA);
    // init: counter and convergence flag to zero, previous energies = current ones
    if (cudaStreamBeginCaptureToGraph(c.stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return fail(SSCF_ERR_CUDA);
    cudaError_t e1 = cudaMemsetAsync(c.d_loop, 0, 16, c.stream);
    cudaError_t e2 = cudaMemcpyAsync(c.d_cl_Eprev, c.d_cl_E, (size_t)c.n_clusters * 8, cudaMemcpyDeviceToDevice,
                                     c.stream);
    cudaGraph_t gg = nullptr;
    if (cudaStreamEndCapture(c.stream, &gg) != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(SSCF_ERR_CUDA);
    size_t n_nodes = 0;
    if (cudaGraphGetNodes(g, nullptr, &n_nodes) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    std::vector<cudaGraphNode_t> deps(n_nodes);
    if (n_nodes && cudaGraphGetNodes(g, deps.data(), &n_nodes) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond;
    if (cudaGraphAddNode(&cond, g, deps.data(), nullptr, n_nodes, &cp) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // body: one SCC iteration and the convergence test
    if (cudaStreamBeginCaptureToGraph(c.stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return fail(SSCF_ERR_CUDA);
    st = step_device(c);
    if (st == SSCF_OK) {
        k_scc_loop_test<<<1, 256, 0, c.stream>>>(c.n_clusters, c.d_cl_E, c.d_cl_Eprev, c.d_cl_dq, dq_tol, e_tol,
                                                 max_iter, c.d_loop, &c.d_sc->err, handle);
        c.n_launch += 1;
        if (cudaGetLastError() != cudaSuccess) st = SSCF_ERR_CUDA;
    }
    cudaGraph_t gb = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c.stream, &gb);
    body_launches = c.n_launch - l0;
    if (st != SSCF_OK) return fail(st);
    if (ce != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (c.cur != cur0) return fail(SSCF_ERR_STATE);
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    if (cudaGraphLaunch(exec, c.stream) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    int loop[2] = {0, 0};
    if (cudaMemcpyAsync(loop, c.d_loop, 8, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess) return fail(SSCF_ERR_CUDA);
    st = sync_scalars(c);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(g);
    c.prof = prof;
    c.n_launch = l0 + (long long)loop[0] * body_launches;
    if (st != SSCF_OK) return st;
    c.iteration += loop[0];
    if (last) {
        last->energy = c.h_sc->energy;
        last->dq_max = c.h_sc->dq_max;
        last->dE = c.have_e_prev ? c.h_sc->energy - c.e_prev : c.h_sc->energy;
        last->max_fov = c.h_sc->max_fov;
        last->eta = c.h_sc->eta;
        last->n_rot = (int64_t)c.h_sc->n_rot;
        last->n_combo = (int64_t)c.h_sc->n_combo;
        last->nnz_c = (int64_t)c.h_sc->tiles[0] * kTileVals;
        last->nnz_occ = (int64_t)c.h_sc->tiles[1] * kTileVals;
        last->launches = (int64_t)body_launches;
        last->upd_rot = (int64_t)c.h_sc->upd[0];
        last->upd_combo = (int64_t)c.h_sc->upd[1];
        last->iteration = c.iteration;
    }
    if (!std::isfinite(c.h_sc->energy)) return SSCF_ERR_NONFINITE;
    c.e_prev = c.h_sc->energy;
    c.have_e_prev = true;
    *converged = loop[1] != 0;
    return SSCF_OK;
}

// The two-stage SCF (Section "Sparsity and numerical accuracy"), or, from the
// MOs already in the context, the user stage alone.
static int run_impl(sscf_ctx* h, sscf_step_info* info, bool from_current) {
    Ctx& c = h->c;
    const double eps_u = c.prm.eps, dq_u = c.prm.dq_tol, e_u = c.prm.e_tol;
    if (from_current) {
        if (!c.have_guess) return SSCF_ERR_STATE;
    } else {
        CKS(sscf_guess(h));
    }
    struct Stage {
        double eps, dq, e;
    } stages[2] = {{1e-3, 1e-1, INFINITY}, {eps_u, dq_u, e_u}};
    sscf_step_info last{};
    bool converged = false;
    for (int s = from_current ? 1 : 0; s < 2; ++s) {
        if (c.prm.eps != stages[s].eps) drop_graph(c);
        c.prm.eps = stages[s].eps;
        CKS(sscf_orthonormalise(h, SSCF_ORTHO_ALL, 200, nullptr, nullptr));
        if (s == 0 || from_current) CKS(sscf_reset_charges(h, nullptr));
        converged = false;
        if (c.use_graph && c.prm.max_scc > 0) {
            int st = stage_in_graph(c, stages[s].dq, stages[s].e, c.prm.max_scc, &converged, &last);
            if (st != SSCF_ERR_STATE) {
                CKS(st);
                continue;
            }
            // the captured iteration does not end in the buffer it starts from: host loop
        }
        std::vector<double> e_prev(c.n_clusters), e_now(c.n_clusters), dq_now(c.n_clusters);
        CKS(sscf_get_cluster_results(h, e_prev.data(), nullptr, nullptr));
        for (int it = 0; it < c.prm.max_scc; ++it) {
            CKS(sscf_step(h, &last));
            CKS(sscf_get_cluster_results(h, e_now.data(), dq_now.data(), nullptr));
            double de = 0.0, dq = 0.0;
            for (int k = 0; k < c.n_clusters; ++k) {
                de = std::max(de, std::fabs(e_now[k] - e_prev[k]));
                dq = std::max(dq, dq_now[k]);
            }
            e_prev = e_now;
            if (dq <= stages[s].dq && de <= stages[s].e) {
                converged = true;
                break;
            }
        }
    }
    if (c.prm.eps != eps_u) drop_graph(c);
    c.prm.eps = eps_u;
    c.prm.dq_tol = dq_u;
    c.prm.e_tol = e_u;
    // mixed precision: the SCC stages orthonormalised to max(eps / 100, 32 u_fp32);
    // the MOs are widened to FP64 and the occupied ones polished to eps / 100
    // before the final charges and energy (the context stays FP64)
    if (c.prec == SSCF_MIXED) CKS(sscf_set_precision(h, SSCF_FP64));
    CKS(sscf_orthonormalise(h, SSCF_ORTHO_OCC, 200, nullptr, nullptr));
    double E = 0.0;
    CK(cudaMemsetAsync(c.d_sc, 0, sizeof(unsigned), c.stream));
    CKS(density_async(c, false));
    CKS(finish_charges(c, nullptr, &E, nullptr));
    last.energy = E;
    if (info) *info = last;
    return converged ? SSCF_OK : SSCF_ERR_NOT_CONVERGED;
}

int sscf_run(sscf_ctx* h, sscf_step_info* info) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    return run_impl(h, info, false);
}

int sscf_run_from_current(sscf_ctx* h, sscf_step_info* info) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    return run_impl(h, info, true);
}

}  // extern "C"
