// Constrained k-means grouping of molecules into MO groups (Section "Defining
// neighbouring lists of atoms and MOs").
//
// Centres start on a grid spread over the bounding box of the molecules; each
// iteration links every molecule to a centre with at most n_link molecules per
// centre, then moves every centre to the centroid of its molecules, until the
// average move falls below tol or max_iter iterations ran.
//
// The paper links atoms in list order (one OpenMP lock per centre) and evens
// out the order dependence by shuffling the centres at every iteration. Here
// the link step is the molecule-proposing deferred-acceptance matching: in
// rounds, every unlinked molecule proposes to its next centre in increasing
// (distance^2, centre index); every centre keeps the n_link candidates (its
// members and the new proposers) with the smallest (distance^2, molecule
// index). The result does not depend on any processing order, so one thread
// per molecule and one per centre compute it without locks, bit for bit the
// same on every run. Squared distances are (dx*dx + dy*dy) + dz*dz with
// explicitly rounded operations (no fused multiply-add).
#include <algorithm>
#include <cmath>
#include <vector>

#include "sscf_internal.h"

namespace sscf {
namespace {

__device__ __forceinline__ double d2_rn(const double* a, const double* b) {
    const double dx = __dsub_rn(b[0], a[0]), dy = __dsub_rn(b[1], a[1]), dz = __dsub_rn(b[2], a[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// (d, i) < (e, j) lexicographically
__device__ __forceinline__ bool lex_less(double d, int i, double e, int j) { return d < e || (d == e && i < j); }

// Every unlinked molecule proposes to its next centre: the smallest
// (distance^2, centre) above the last one it proposed to.
__global__ void k_km_propose(int n, int nc, const double* __restrict__ pos, const double* __restrict__ cen,
                             const int* __restrict__ holder, int* __restrict__ prop, double* __restrict__ last_d,
                             int* __restrict__ last_c, int* __restrict__ n_free) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    if (holder[m] >= 0) {
        prop[m] = -1;
        return;
    }
    const double ld = last_d[m];
    const int lc = last_c[m];
    double bd = INFINITY;
    int bc = -1;
    for (int c = 0; c < nc; ++c) {
        const double d = d2_rn(pos + 3 * m, cen + 3 * c);
        if (lc >= 0 && !lex_less(ld, lc, d, c)) continue;   // at or before the last proposal
        if (bc < 0 || lex_less(d, c, bd, bc)) {
            bd = d;
            bc = c;
        }
    }
    prop[m] = bc;
    last_d[m] = bd;
    last_c[m] = bc;
    atomicAdd(n_free, 1);
}

// Every centre keeps its n_link best candidates (members and new proposers).
template <int kMaxLink>
__global__ void k_km_accept(int n, int nc, int n_link, const double* __restrict__ pos, const double* __restrict__ cen,
                            int* __restrict__ holder, const int* __restrict__ prop) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double kd[kMaxLink];
    int km[kMaxLink];
    int nk = 0;
    for (int m = 0; m < n; ++m) {
        if (holder[m] != c && prop[m] != c) continue;
        const double d = d2_rn(pos + 3 * m, cen + 3 * c);
        if (nk == n_link && !lex_less(d, m, kd[nk - 1], km[nk - 1])) {
            holder[m] = -1;   // rejected (or displaced)
            continue;
        }
        if (nk == n_link) holder[km[nk - 1]] = -1;   // the worst kept one is displaced
        int p = nk < n_link ? nk++ : nk - 1;
        while (p > 0 && lex_less(d, m, kd[p - 1], km[p - 1])) {
            kd[p] = kd[p - 1];
            km[p] = km[p - 1];
            --p;
        }
        kd[p] = d;
        km[p] = m;
        holder[m] = c;
    }
}

// Centroid of every centre's members, summed in increasing molecule index; a
// centre without members keeps its place.
__global__ void k_km_centroids(int n, int nc, const double* __restrict__ pos, const int* __restrict__ holder,
                               const double* __restrict__ cen, double* __restrict__ cen_new) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    int k = 0;
    for (int m = 0; m < n; ++m) {
        if (holder[m] != c) continue;
        s0 = __dadd_rn(s0, pos[3 * m]);
        s1 = __dadd_rn(s1, pos[3 * m + 1]);
        s2 = __dadd_rn(s2, pos[3 * m + 2]);
        ++k;
    }
    if (k == 0) {
        cen_new[3 * c] = cen[3 * c];
        cen_new[3 * c + 1] = cen[3 * c + 1];
        cen_new[3 * c + 2] = cen[3 * c + 2];
    } else {
        cen_new[3 * c] = __ddiv_rn(s0, (double)k);
        cen_new[3 * c + 1] = __ddiv_rn(s1, (double)k);
        cen_new[3 * c + 2] = __ddiv_rn(s2, (double)k);
    }
}

struct Buf {
    std::vector<void*> ptrs;
    ~Buf() {
        for (void* p : ptrs) raw_free(p);
    }
    template <typename T>
    T* get(size_t n) {
        void* p = raw_alloc(n * sizeof(T));
        if (p) ptrs.push_back(p);
        return (T*)p;
    }
};

#define KM_CK(call)                                 \
    do {                                            \
        if ((call) != cudaSuccess) {                \
            cudaGetLastError();                     \
            return SSCF_ERR_CUDA;                   \
        }                                           \
    } while (0)

// Deferred acceptance on the device: every molecule linked, at most n_link per centre.
int link_all(cudaStream_t st, int n, int nc, int n_link, const double* d_pos, const double* d_cen, int* d_holder,
             int* d_prop, double* d_last_d, int* d_last_c, int* d_free) {
    KM_CK(cudaMemsetAsync(d_holder, 0xff, (size_t)n * 4, st));   // -1: unlinked
    KM_CK(cudaMemsetAsync(d_last_c, 0xff, (size_t)n * 4, st));
    const int th = 128;
    // each round links or moves at least one molecule a step down its list: at most n * nc rounds
    for (long long round = 0; round <= (long long)n * nc; ++round) {
        KM_CK(cudaMemsetAsync(d_free, 0, 4, st));
        k_km_propose<<<(n + th - 1) / th, th, 0, st>>>(n, nc, d_pos, d_cen, d_holder, d_prop, d_last_d, d_last_c,
                                                       d_free);
        int n_free = 0;
        KM_CK(cudaMemcpyAsync(&n_free, d_free, 4, cudaMemcpyDeviceToHost, st));
        KM_CK(cudaStreamSynchronize(st));
        if (n_free == 0) return SSCF_OK;
        k_km_accept<kMaxMolPerGroup><<<(nc + th - 1) / th, th, 0, st>>>(n, nc, n_link, d_pos, d_cen, d_holder, d_prop);
        KM_CK(cudaGetLastError());
    }
    return SSCF_ERR_STATE;
}

}  // namespace
}  // namespace sscf

using namespace sscf;

extern "C" int sscf_group_molecules(int n_atoms, const double* xyz, int n_link, int max_iter, double tol,
                                    void* cuda_stream, int* group_of_mol, int* n_groups_out, int* iters_out) {
    if (n_atoms <= 0 || n_atoms % 3 != 0 || !xyz || !group_of_mol) return SSCF_ERR_INVALID_ARG;
    if (n_link < 1 || n_link > kMaxMolPerGroup || max_iter < 0 || !(tol >= 0.0)) return SSCF_ERR_INVALID_ARG;
    const int n = n_atoms / 3;
    std::vector<double> pos(3 * (size_t)n);
    for (int m = 0; m < n; ++m)
        for (int d = 0; d < 3; ++d) {
            pos[3 * (size_t)m + d] = xyz[9 * (size_t)m + d];   // the molecule's first (oxygen) atom
            if (!std::isfinite(pos[3 * (size_t)m + d])) return SSCF_ERR_NONFINITE;
        }
    // centres: a grid over the bounding box, refined along the axis with the
    // largest spacing (lowest axis on ties) until it has ceil(n / n_link) points
    double lo[3], L[3];
    for (int d = 0; d < 3; ++d) {
        double a = pos[d], b = pos[d];
        for (int m = 1; m < n; ++m) {
            a = std::min(a, pos[3 * (size_t)m + d]);
            b = std::max(b, pos[3 * (size_t)m + d]);
        }
        lo[d] = a;
        L[d] = std::max(b - a, 1.0);
    }
    const long long need = ((long long)n + n_link - 1) / n_link;
    long long g[3] = {1, 1, 1};
    while (g[0] * g[1] * g[2] < need) {
        int best = 0;
        for (int d = 1; d < 3; ++d)
            if (L[d] / (double)g[d] > L[best] / (double)g[best]) best = d;
        g[best]++;
    }
    const int nc = (int)(g[0] * g[1] * g[2]);
    std::vector<double> cen(3 * (size_t)nc), cen_new(3 * (size_t)nc);
    {
        size_t c = 0;
        for (long long k = 0; k < g[2]; ++k)
            for (long long j = 0; j < g[1]; ++j)
                for (long long i = 0; i < g[0]; ++i, ++c) {
                    const long long idx[3] = {i, j, k};
                    for (int d = 0; d < 3; ++d)
                        cen[3 * c + d] = lo[d] + ((double)(2 * idx[d] + 1) * L[d]) / (double)(2 * g[d]);
                }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Buf buf;
    double* d_pos = buf.get<double>(3 * (size_t)n);
    double* d_cen = buf.get<double>(3 * (size_t)nc);
    double* d_cen_new = buf.get<double>(3 * (size_t)nc);
    int* d_holder = buf.get<int>(n);
    int* d_prop = buf.get<int>(n);
    double* d_last_d = buf.get<double>(n);
    int* d_last_c = buf.get<int>(n);
    int* d_free = buf.get<int>(1);
    if (!d_pos || !d_cen || !d_cen_new || !d_holder || !d_prop || !d_last_d || !d_last_c || !d_free)
        return SSCF_ERR_OOM;
    KM_CK(cudaMemcpyAsync(d_pos, pos.data(), pos.size() * 8, cudaMemcpyHostToDevice, st));
    KM_CK(cudaMemcpyAsync(d_cen, cen.data(), cen.size() * 8, cudaMemcpyHostToDevice, st));
    int s = link_all(st, n, nc, n_link, d_pos, d_cen, d_holder, d_prop, d_last_d, d_last_c, d_free);
    if (s != SSCF_OK) return s;
    int it = 0;
    const int th = 128;
    for (it = 1; it <= max_iter; ++it) {
        k_km_centroids<<<(nc + th - 1) / th, th, 0, st>>>(n, nc, d_pos, d_holder, d_cen, d_cen_new);
        KM_CK(cudaGetLastError());
        KM_CK(cudaMemcpyAsync(cen_new.data(), d_cen_new, cen_new.size() * 8, cudaMemcpyDeviceToHost, st));
        KM_CK(cudaStreamSynchronize(st));
        double moved = 0.0;
        for (int c = 0; c < nc; ++c) {
            const double dx = cen_new[3 * c] - cen[3 * c], dy = cen_new[3 * c + 1] - cen[3 * c + 1],
                         dz = cen_new[3 * c + 2] - cen[3 * c + 2];
            const double xx = dx * dx, yy = dy * dy, zz = dz * dz;
            const double t = xx + yy;
            moved += std::sqrt(t + zz);
        }
        std::swap(cen, cen_new);
        std::swap(d_cen, d_cen_new);
        s = link_all(st, n, nc, n_link, d_pos, d_cen, d_holder, d_prop, d_last_d, d_last_c, d_free);
        if (s != SSCF_OK) return s;
        if (moved / nc < tol) break;
    }
    if (it > max_iter) it = max_iter;
    std::vector<int> holder(n);
    KM_CK(cudaMemcpyAsync(holder.data(), d_holder, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    KM_CK(cudaStreamSynchronize(st));
    std::vector<int> remap(nc, -1);
    for (int m = 0; m < n; ++m) {
        if (holder[m] < 0 || holder[m] >= nc) return SSCF_ERR_STATE;
        remap[holder[m]] = 0;
    }
    int G = 0;
    for (int c = 0; c < nc; ++c)
        if (remap[c] == 0) remap[c] = G++;
    for (int m = 0; m < n; ++m) group_of_mol[m] = remap[holder[m]];
    if (n_groups_out) *n_groups_out = G;
    if (iters_out) *iters_out = it;
    return SSCF_OK;
}
