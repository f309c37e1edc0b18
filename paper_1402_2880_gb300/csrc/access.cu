// State access of libsscf: dense copies for tests and checkpoints, charges,
// the group colouring and the last pair list.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sscf_internal.h"

using namespace sscf;

namespace {

#define CKA(call)                                  \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            cudaGetLastError();                    \
            return SSCF_ERR_CUDA;                  \
        }                                          \
    } while (0)

template <typename T>
void widen(const std::vector<unsigned char>& raw, std::vector<double>& out) {
    const T* p = reinterpret_cast<const T*>(raw.data());
    out.resize(raw.size() / sizeof(T));
    for (size_t i = 0; i < out.size(); ++i) out[i] = (double)p[i];
}

int fetch_values(Ctx& c, const void* dptr, size_t n, std::vector<double>& out) {
    std::vector<unsigned char> raw(n * c.tsize);
    CKA(cudaStreamSynchronize(c.stream));
    CKA(cudaMemcpy(raw.data(), dptr, raw.size(), cudaMemcpyDeviceToHost));
    if (c.prec == SSCF_FP64)
        widen<double>(raw, out);
    else
        widen<float>(raw, out);
    return SSCF_OK;
}

// Restart of C: packed tiles (FP64, row block after row block) scattered into
// the padded row layout of buffer 0, converted to the storage type.
template <typename T>
__global__ void k_scatter_tiles(int cap, const long long* __restrict__ row_off, const int* __restrict__ nt,
                                const int* __restrict__ tiles, const double* __restrict__ vals,
                                int* __restrict__ c_tile, T* __restrict__ c_val) {
    const int r = blockIdx.x;
    const long long o = row_off[r];
    const int n = nt[r];
    for (int s = threadIdx.x; s < n; s += blockDim.x) c_tile[(size_t)r * cap + s] = tiles[o + s];
    const double* src = vals + o * kTileVals;
    T* dst = c_val + (size_t)r * cap * kTileVals;
    for (long long i = threadIdx.x; i < (long long)n * kTileVals; i += blockDim.x) dst[i] = (T)src[i];
}

// Non-finite check of the staged values (before anything of the context is written).
__global__ void k_check_finite(long long n, const double* __restrict__ v, unsigned* __restrict__ bad) {
    unsigned b = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b |= isfinite(v[i]) ? 0u : 1u;
    if (__any_sync(0xffffffffu, b != 0u) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// Staging buffer of the restart (kept and grown as needed).
int stage(Ctx& c, size_t bytes, unsigned char** out) {
    if (c.stage_bytes < bytes) {
        dev_release(&c, c.d_stage);
        c.d_stage = nullptr;
        c.stage_bytes = 0;
        void* p = nullptr;
        int s = dev_alloc(&c, &p, bytes);
        if (s != SSCF_OK) return s;
        c.d_stage = (unsigned char*)p;
        c.stage_bytes = bytes;
    }
    *out = c.d_stage;
    return SSCF_OK;
}

}  // namespace

extern "C" {

int sscf_get_C_dense(sscf_ctx* h, double* C) {
    if (!h || !C) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const int b = c.cur;
    std::vector<int> nt(c.n_mol), tiles((size_t)c.n_mol * c.cap);
    CKA(cudaStreamSynchronize(c.stream));
    CKA(cudaMemcpy(nt.data(), c.d_c_nt[b], nt.size() * 4, cudaMemcpyDeviceToHost));
    CKA(cudaMemcpy(tiles.data(), c.d_c_tile[b], tiles.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<double> v;
    int s = fetch_values(c, c.d_c_val[b], (size_t)c.n_mol * c.cap * kTileVals, v);
    if (s != SSCF_OK) return s;
    std::memset(C, 0, sizeof(double) * (size_t)c.n_ao * c.n_mo);
    for (int r = 0; r < c.n_mol; ++r)
        for (int sl = 0; sl < nt[r]; ++sl) {
            const int t = tiles[(size_t)r * c.cap + sl];
            if (t < 0 || t >= c.n_tiles) return SSCF_ERR_STATE;
            for (int k = 0; k < 6; ++k)
                for (int col = 0; col < c.h_tile_nmo[t]; ++col)
                    C[(size_t)(6 * r + k) * c.n_mo + c.h_tile_mo0[t] + col] =
                        v[(((size_t)r * c.cap + sl) * 6 + k) * 16 + col];
        }
    return SSCF_OK;
}

int sscf_set_C_dense(sscf_ctx* h, const double* C) {
    if (!h || !C) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    c.cur = 0;
    std::vector<int> nt(c.n_mol, 0), tiles((size_t)c.n_mol * c.cap, 0);
    std::vector<double> v((size_t)c.n_mol * c.cap * kTileVals, 0.0);
    for (int r = 0; r < c.n_mol; ++r) {
        int n = 0;
        for (int t = 0; t < c.n_tiles; ++t) {
            bool nz = false;
            for (int k = 0; k < 6 && !nz; ++k)
                for (int col = 0; col < c.h_tile_nmo[t] && !nz; ++col) {
                    double x = C[(size_t)(6 * r + k) * c.n_mo + c.h_tile_mo0[t] + col];
                    if (!std::isfinite(x)) return SSCF_ERR_NONFINITE;
                    nz = x != 0.0;
                }
            if (!nz) continue;
            if (n >= c.cap) return SSCF_ERR_CAPACITY;
            tiles[(size_t)r * c.cap + n] = t;
            for (int k = 0; k < 6; ++k)
                for (int col = 0; col < c.h_tile_nmo[t]; ++col)
                    v[(((size_t)r * c.cap + n) * 6 + k) * 16 + col] =
                        C[(size_t)(6 * r + k) * c.n_mo + c.h_tile_mo0[t] + col];
            ++n;
        }
        nt[r] = n;
    }
    CKA(cudaStreamSynchronize(c.stream));
    CKA(cudaMemcpy(c.d_c_nt[0], nt.data(), nt.size() * 4, cudaMemcpyHostToDevice));
    CKA(cudaMemcpy(c.d_c_tile[0], tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice));
    if (c.prec == SSCF_FP64) {
        CKA(cudaMemcpy(c.d_c_val[0], v.data(), v.size() * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        CKA(cudaMemcpy(c.d_c_val[0], f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    }
    c.have_guess = true;
    return SSCF_OK;
}

// Checkpoint of C in its stored form: per row block the sorted tile ids and
// their 6x16 values (FP64 on the host in both precisions).
int sscf_get_C_tiles(sscf_ctx* h, int32_t* nt_out, int32_t* tiles_out, double* vals_out, int64_t* n_stored) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const int b = c.cur;
    std::vector<int> nt(c.n_mol);
    CKA(cudaStreamSynchronize(c.stream));
    CKA(cudaMemcpy(nt.data(), c.d_c_nt[b], nt.size() * 4, cudaMemcpyDeviceToHost));
    int64_t tot = 0;
    for (int r = 0; r < c.n_mol; ++r) {
        if (nt[r] < 0 || nt[r] > c.cap) return SSCF_ERR_STATE;
        tot += nt[r];
    }
    if (n_stored) *n_stored = tot;
    if (nt_out) std::copy(nt.begin(), nt.end(), nt_out);
    if (!tiles_out && !vals_out) return SSCF_OK;
    std::vector<unsigned char> raw((size_t)c.cap * kTileVals * c.tsize);
    int64_t off = 0;
    for (int r = 0; r < c.n_mol; ++r) {
        if (nt[r] == 0) continue;
        if (tiles_out)
            CKA(cudaMemcpy(tiles_out + off, c.d_c_tile[b] + (size_t)r * c.cap, (size_t)nt[r] * 4,
                           cudaMemcpyDeviceToHost));
        if (vals_out) {
            const size_t n = (size_t)nt[r] * kTileVals;
            CKA(cudaMemcpy(raw.data(), (const unsigned char*)c.d_c_val[b] + (size_t)r * c.cap * kTileVals * c.tsize,
                           n * c.tsize, cudaMemcpyDeviceToHost));
            double* dst = vals_out + off * kTileVals;
            if (c.prec == SSCF_FP64)
                std::memcpy(dst, raw.data(), n * 8);
            else
                for (size_t i = 0; i < n; ++i) dst[i] = (double)((const float*)raw.data())[i];
        }
        off += nt[r];
    }
    return SSCF_OK;
}

int sscf_set_C_tiles(sscf_ctx* h, const int32_t* nt_in, const int32_t* tiles_in, const double* vals_in) {
    if (!h || !nt_in) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    std::vector<int> group_cl(c.n_groups, 0);
    for (int m = 0; m < c.n_mol; ++m) group_cl[c.h_mol_group[m]] = c.h_mol_cluster[m];
    int64_t tot = 0;
    for (int r = 0; r < c.n_mol; ++r) {
        if (nt_in[r] < 0) return SSCF_ERR_INVALID_ARG;
        if (nt_in[r] > c.cap) return SSCF_ERR_CAPACITY;
        tot += nt_in[r];
    }
    if (tot > 0 && (!tiles_in || !vals_in)) return SSCF_ERR_INVALID_ARG;
    int64_t off = 0;
    for (int r = 0; r < c.n_mol; ++r) {   // validate everything before touching the device
        for (int s = 0; s < nt_in[r]; ++s) {
            const int t = tiles_in[off + s];
            if (t < 0 || t >= c.n_tiles || (s > 0 && t <= tiles_in[off + s - 1])) return SSCF_ERR_INVALID_ARG;
            if (group_cl[c.h_tile_group[t]] != c.h_mol_cluster[r]) return SSCF_ERR_INVALID_ARG;
        }
        off += nt_in[r];
    }
    // one bulk copy of the packed arrays, a finiteness check on the device, then a
    // scatter kernel into the padded rows
    std::vector<long long> row_off(c.n_mol);
    off = 0;
    for (int r = 0; r < c.n_mol; ++r) {
        row_off[r] = off;
        off += nt_in[r];
    }
    const size_t b_off = (size_t)c.n_mol * 8, b_nt = (size_t)c.n_mol * 4, b_tiles = ((size_t)tot * 4 + 15) & ~(size_t)15;
    const size_t b_vals = (size_t)tot * kTileVals * 8;
    unsigned char* st = nullptr;
    int s = stage(c, b_off + ((b_nt + 15) & ~(size_t)15) + b_tiles + b_vals + 16, &st);
    if (s != SSCF_OK) return s;
    unsigned* d_bad = (unsigned*)(st + b_off + ((b_nt + 15) & ~(size_t)15) + b_tiles + b_vals);
    long long* d_off = (long long*)st;
    int* d_nt = (int*)(st + b_off);
    int* d_tiles = (int*)(st + b_off + ((b_nt + 15) & ~(size_t)15));
    double* d_vals = (double*)(st + b_off + ((b_nt + 15) & ~(size_t)15) + b_tiles);
    CKA(cudaMemcpyAsync(d_off, row_off.data(), b_off, cudaMemcpyHostToDevice, c.stream));
    CKA(cudaMemcpyAsync(d_nt, nt_in, b_nt, cudaMemcpyHostToDevice, c.stream));
    CKA(cudaMemsetAsync(d_bad, 0, 4, c.stream));
    if (tot > 0) {
        CKA(cudaMemcpyAsync(d_tiles, tiles_in, (size_t)tot * 4, cudaMemcpyHostToDevice, c.stream));
        CKA(cudaMemcpyAsync(d_vals, vals_in, b_vals, cudaMemcpyHostToDevice, c.stream));
        const long long nv = tot * kTileVals;
        const int blocks = (int)std::min<long long>((nv + 255) / 256, (long long)c.n_sm * 8);
        k_check_finite<<<blocks, 256, 0, c.stream>>>(nv, d_vals, d_bad);
        c.n_launch += 1;
        CKA(cudaGetLastError());
        unsigned bad = 0;
        CKA(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, c.stream));
        CKA(cudaStreamSynchronize(c.stream));
        if (bad) return SSCF_ERR_NONFINITE;
    }
    if (c.prec == SSCF_FP64)
        k_scatter_tiles<double><<<c.n_mol, 256, 0, c.stream>>>(c.cap, d_off, d_nt, d_tiles, d_vals, c.d_c_tile[0],
                                                               (double*)c.d_c_val[0]);
    else
        k_scatter_tiles<float><<<c.n_mol, 256, 0, c.stream>>>(c.cap, d_off, d_nt, d_tiles, d_vals, c.d_c_tile[0],
                                                              (float*)c.d_c_val[0]);
    c.n_launch += 1;
    CKA(cudaGetLastError());
    CKA(cudaMemcpyAsync(c.d_c_nt[0], d_nt, b_nt, cudaMemcpyDeviceToDevice, c.stream));
    CKA(cudaStreamSynchronize(c.stream));
    c.cur = 0;
    c.have_guess = true;
    return SSCF_OK;
}

// Rows (AO indices) of C, dense over all MOs: out is n x n_mo, row-major.
int sscf_get_C_rows(sscf_ctx* h, int n, const int* rows, double* out) {
    if (!h || n < 0 || (n > 0 && (!rows || !out))) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const int b = c.cur;
    CKA(cudaStreamSynchronize(c.stream));
    std::memset(out, 0, sizeof(double) * (size_t)n * c.n_mo);
    std::vector<int> tiles(c.cap);
    std::vector<unsigned char> raw((size_t)c.cap * kTileVals * c.tsize);
    for (int i = 0; i < n; ++i) {
        const int mu = rows[i];
        if (mu < 0 || mu >= c.n_ao) return SSCF_ERR_INVALID_ARG;
        const int r = mu / 6, k = mu % 6;
        int nt = 0;
        CKA(cudaMemcpy(&nt, c.d_c_nt[b] + r, 4, cudaMemcpyDeviceToHost));
        if (nt < 0 || nt > c.cap) return SSCF_ERR_STATE;
        CKA(cudaMemcpy(tiles.data(), c.d_c_tile[b] + (size_t)r * c.cap, (size_t)nt * 4, cudaMemcpyDeviceToHost));
        CKA(cudaMemcpy(raw.data(), (const unsigned char*)c.d_c_val[b] + (size_t)r * c.cap * kTileVals * c.tsize,
                       (size_t)nt * kTileVals * c.tsize, cudaMemcpyDeviceToHost));
        for (int s = 0; s < nt; ++s) {
            const int t = tiles[s];
            for (int col = 0; col < c.h_tile_nmo[t]; ++col) {
                const size_t e = (size_t)s * kTileVals + k * 16 + col;
                const double v = c.prec == SSCF_FP64 ? ((const double*)raw.data())[e] : (double)((const float*)raw.data())[e];
                out[(size_t)i * c.n_mo + c.h_tile_mo0[t] + col] = v;
            }
        }
    }
    return SSCF_OK;
}

// Columns (MO indices) of C, dense over all AOs: out is n_ao x n, row-major.
// Each stored tile a column needs is copied once per row block.
int sscf_get_C_cols(sscf_ctx* h, int n, const int* cols, double* out) {
    if (!h || n < 0 || (n > 0 && (!cols || !out))) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const int b = c.cur;
    std::vector<int> mo_tile(c.n_mo);
    for (int t = 0; t < c.n_tiles; ++t)
        for (int k = 0; k < c.h_tile_nmo[t]; ++k) mo_tile[c.h_tile_mo0[t] + k] = t;
    std::vector<int> want;   // distinct tiles, sorted
    for (int i = 0; i < n; ++i) {
        if (cols[i] < 0 || cols[i] >= c.n_mo) return SSCF_ERR_INVALID_ARG;
        want.push_back(mo_tile[cols[i]]);
    }
    std::sort(want.begin(), want.end());
    want.erase(std::unique(want.begin(), want.end()), want.end());
    std::vector<int> nt(c.n_mol), tiles((size_t)c.n_mol * c.cap);
    CKA(cudaStreamSynchronize(c.stream));
    CKA(cudaMemcpy(nt.data(), c.d_c_nt[b], nt.size() * 4, cudaMemcpyDeviceToHost));
    CKA(cudaMemcpy(tiles.data(), c.d_c_tile[b], tiles.size() * 4, cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(double) * (size_t)c.n_ao * n);
    std::vector<unsigned char> raw(kTileVals * c.tsize);
    for (int r = 0; r < c.n_mol; ++r) {
        if (nt[r] < 0 || nt[r] > c.cap) return SSCF_ERR_STATE;
        const int* tr = tiles.data() + (size_t)r * c.cap;
        for (int t : want) {
            const int* p = std::lower_bound(tr, tr + nt[r], t);
            if (p == tr + nt[r] || *p != t) continue;
            const size_t s = p - tr;
            CKA(cudaMemcpy(raw.data(), (const unsigned char*)c.d_c_val[b] + ((size_t)r * c.cap + s) * kTileVals * c.tsize,
                           raw.size(), cudaMemcpyDeviceToHost));
            for (int i = 0; i < n; ++i) {
                if (mo_tile[cols[i]] != t) continue;
                const int col = cols[i] - c.h_tile_mo0[t];
                for (int k = 0; k < 6; ++k) {
                    const size_t e = (size_t)k * 16 + col;
                    out[(size_t)(6 * r + k) * n + i] =
                        c.prec == SSCF_FP64 ? ((const double*)raw.data())[e] : (double)((const float*)raw.data())[e];
                }
            }
        }
    }
    return SSCF_OK;
}

// Entries F_ov(i, j) of the last transform (0 outside the kept blocks), i
// occupied, j virtual (global MO indices).
int sscf_get_F_entries(sscf_ctx* h, int n, const int* i_mo, const int* j_mo, double* out) {
    if (!h || n < 0 || (n > 0 && (!i_mo || !j_mo || !out))) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    std::vector<int> g_of_occ(c.n_occ), g_of_virt(c.n_mo - c.n_occ);
    for (int g = 0; g < c.n_groups; ++g) {
        for (int k = 0; k < 4 * c.h_group_nmol[g]; ++k) g_of_occ[c.h_group_occ0[g] + k] = g;
        for (int k = 0; k < 2 * c.h_group_nmol[g]; ++k) g_of_virt[c.h_group_virt0[g] - c.n_occ + k] = g;
    }
    CKA(cudaStreamSynchronize(c.stream));
    std::vector<unsigned char> raw(c.tsize);
    for (int q = 0; q < n; ++q) {
        const int i = i_mo[q], j = j_mo[q];
        if (i < 0 || i >= c.n_occ || j < c.n_occ || j >= c.n_mo) return SSCF_ERR_INVALID_ARG;
        const int A = g_of_occ[i], B = g_of_virt[j - c.n_occ];
        const int* lo = c.h_gnb_col.data() + c.h_gnb_ptr[A];
        const int* hi = c.h_gnb_col.data() + c.h_gnb_ptr[A + 1];
        const int* p = std::lower_bound(lo, hi, B);
        out[q] = 0.0;
        if (p == hi || *p != B) continue;
        const int e = c.h_gnb_ptr[A] + (int)(p - lo);
        const int il = i - c.h_group_occ0[A], jl = j - c.h_group_virt0[B];
        const int tp = c.h_rot_blk_tp0[e] + (il / 16) * c.h_group_nvt[B] + jl / 16;
        const size_t off = ((size_t)tp * 256 + (il % 16) * 16 + jl % 16) * c.tsize;
        CKA(cudaMemcpy(raw.data(), (const unsigned char*)c.d_F + off, c.tsize, cudaMemcpyDeviceToHost));
        out[q] = c.prec == SSCF_FP64 ? *(const double*)raw.data() : (double)*(const float*)raw.data();
    }
    return SSCF_OK;
}

// The molecule-pair blocks of H (current), H0 and S: pairs (m, n) into
// mn (2 * n_mp ints) and 36 values per block into each non-NULL array
// (n_mp * 36 doubles, row-major 6 x 6). n_mp_out receives the count; call
// with NULL arrays first to size them.
int sscf_get_blocks(sscf_ctx* h, int* mn, double* H, double* H0, double* S, int64_t* n_mp_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (n_mp_out) *n_mp_out = c.n_mp;
    if (mn)
        for (int m = 0; m < c.n_mol; ++m)
            for (int e = c.h_mp_ptr[m]; e < c.h_mp_ptr[m + 1]; ++e) {
                mn[2 * e] = m;
                mn[2 * e + 1] = c.h_mp_col[e];
            }
    if (H) {
        std::vector<double> v;
        int s = fetch_values(c, c.d_Hb, (size_t)c.n_mp * 36, v);
        if (s != SSCF_OK) return s;
        std::memcpy(H, v.data(), v.size() * 8);
    }
    CKA(cudaStreamSynchronize(c.stream));
    if (H0) CKA(cudaMemcpy(H0, c.d_H0b, (size_t)c.n_mp * 36 * 8, cudaMemcpyDeviceToHost));
    if (S) CKA(cudaMemcpy(S, c.d_Sb, (size_t)c.n_mp * 36 * 8, cudaMemcpyDeviceToHost));
    return SSCF_OK;
}

int sscf_get_H_dense(sscf_ctx* h, double* H, double* H0, double* S) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    std::vector<double> hv, h0((size_t)c.n_mp * 36), sv((size_t)c.n_mp * 36);
    int s = fetch_values(c, c.d_Hb, (size_t)c.n_mp * 36, hv);
    if (s != SSCF_OK) return s;
    CKA(cudaMemcpy(h0.data(), c.d_H0b, h0.size() * 8, cudaMemcpyDeviceToHost));
    CKA(cudaMemcpy(sv.data(), c.d_Sb, sv.size() * 8, cudaMemcpyDeviceToHost));
    const size_t N = (size_t)c.n_ao;
    for (double* M : {H, H0, S})
        if (M) std::memset(M, 0, sizeof(double) * N * N);
    for (int m = 0; m < c.n_mol; ++m)
        for (int k = c.h_mp_ptr[m]; k < c.h_mp_ptr[m + 1]; ++k) {
            const int n = c.h_mp_col[k];
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    const size_t d = (size_t)(6 * m + i) * N + 6 * n + j;
                    const size_t e = (size_t)k * 36 + i * 6 + j;
                    if (H) H[d] = hv[e];
                    if (H0) H0[d] = h0[e];
                    if (S) S[d] = sv[e];
                }
        }
    return SSCF_OK;
}

int sscf_get_F_dense(sscf_ctx* h, double* F_ov, double* F_diag) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const int nv = c.n_mo - c.n_occ;
    if (F_ov) {
        std::vector<double> f;
        int s = fetch_values(c, c.d_F, (size_t)std::max(c.n_rot_tp, 1) * 256, f);
        if (s != SSCF_OK) return s;
        std::memset(F_ov, 0, sizeof(double) * (size_t)c.n_occ * nv);
        for (int e = 0; e < c.n_gnb; ++e) {
            const int A = c.h_gnb_row[e], B = c.h_gnb_col[e];
            const int no = 4 * c.h_group_nmol[A], nvb = 2 * c.h_group_nmol[B];
            for (int i = 0; i < no; ++i)
                for (int j = 0; j < nvb; ++j) {
                    const int tp = c.h_rot_blk_tp0[e] + (i / 16) * c.h_group_nvt[B] + j / 16;
                    F_ov[(size_t)(c.h_group_occ0[A] + i) * nv + (c.h_group_virt0[B] - c.n_occ + j)] =
                        f[(size_t)tp * 256 + (i % 16) * 16 + j % 16];
                }
        }
    }
    if (F_diag) {
        CKA(cudaStreamSynchronize(c.stream));
        CKA(cudaMemcpy(F_diag, c.d_Fd, (size_t)c.n_mo * 8, cudaMemcpyDeviceToHost));
    }
    return SSCF_OK;
}

// sigma = C^T S C of the last orthonormalisation pass (before normalisation),
// dense over the pass's MOs: n_occ x n_occ after an occupied pass, n_mo x n_mo
// after a pass over all MOs; zero off the kept blocks. The kernels read the
// entries (i, j) with i before j in the pass order (lower group, or lower
// local index inside one group); both halves hold those.
int sscf_get_overlap_dense(sscf_ctx* h, double* sigma, int* n_out) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.last_sched_kind != 2) return SSCF_ERR_STATE;
    const int w = c.last_ortho_which;
    const int n = w == 1 ? c.n_occ : c.n_mo;
    if (n_out) *n_out = n;
    if (!sigma) return SSCF_OK;
    std::vector<double> v;
    int s = fetch_values(c, c.d_sig, (size_t)std::max(c.n_ort_tp[w], 1) * 256, v);
    if (s != SSCF_OK) return s;
    std::memset(sigma, 0, sizeof(double) * (size_t)n * n);
    auto side = [&](int g, int* t) {
        int k = 0;
        for (int i = 0; i < c.h_group_not[g]; ++i) t[k++] = c.h_group_ot0[g] + i;
        if (w == 0)
            for (int i = 0; i < c.h_group_nvt[g]; ++i) t[k++] = c.h_group_vt0[g] + i;
        return k;
    };
    for (int e = 0; e < c.n_gnb; ++e) {
        const int A = c.h_gnb_row[e], B = c.h_gnb_col[e];
        if (A > B) continue;
        int ta[3], tb[3];
        const int na = side(A, ta), nb = side(B, tb);
        for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j) {
                const int tp = c.h_ort_blk_tp[w][(size_t)e * 9 + i * 3 + j];
                if (tp < 0) continue;
                for (int ca = 0; ca < c.h_tile_nmo[ta[i]]; ++ca)
                    for (int cb = 0; cb < c.h_tile_nmo[tb[j]]; ++cb) {
                        if (A == B && i == j && cb < ca) continue;
                        const size_t gi = (size_t)c.h_tile_mo0[ta[i]] + ca, gj = (size_t)c.h_tile_mo0[tb[j]] + cb;
                        const double x = v[(size_t)tp * 256 + ca * 16 + cb];
                        sigma[gi * n + gj] = x;
                        sigma[gj * n + gi] = x;
                    }
            }
    }
    return SSCF_OK;
}

int sscf_get_charges(sscf_ctx* h, double* q_prev, double* dq_in, double* Q_in) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    CKA(cudaStreamSynchronize(c.stream));
    const size_t n = (size_t)c.n_atoms * 8;
    if (q_prev) CKA(cudaMemcpy(q_prev, c.d_q_prev, n, cudaMemcpyDeviceToHost));
    if (dq_in) CKA(cudaMemcpy(dq_in, c.d_dq_in, n, cudaMemcpyDeviceToHost));
    if (Q_in) CKA(cudaMemcpy(Q_in, c.d_Q_in, n, cudaMemcpyDeviceToHost));
    return SSCF_OK;
}

int sscf_set_charges(sscf_ctx* h, const double* q_prev, const double* dq_in, const double* Q_in) {
    if (!h) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    CKA(cudaStreamSynchronize(c.stream));
    const size_t n = (size_t)c.n_atoms * 8;
    for (const double* p : {q_prev, dq_in, Q_in})
        if (p)
            for (int a = 0; a < c.n_atoms; ++a)
                if (!std::isfinite(p[a])) return SSCF_ERR_NONFINITE;
    if (q_prev) CKA(cudaMemcpy(c.d_q_prev, q_prev, n, cudaMemcpyHostToDevice));
    if (dq_in) CKA(cudaMemcpy(c.d_dq_in, dq_in, n, cudaMemcpyHostToDevice));
    if (Q_in) CKA(cudaMemcpy(c.d_Q_in, Q_in, n, cudaMemcpyHostToDevice));
    return SSCF_OK;
}

int sscf_get_colouring(sscf_ctx* h, int* colour) {
    if (!h || !colour) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    const size_t G = (size_t)c.n_groups;
    for (size_t i = 0; i < G * G; ++i) colour[i] = -1;
    for (int e = 0; e < c.n_gnb; ++e) colour[(size_t)c.h_gnb_row[e] * G + c.h_gnb_col[e]] = c.h_gnb_colour[e];
    return SSCF_OK;
}

int sscf_get_pairs(sscf_ctx* h, int64_t capacity, int32_t* colour_out, int32_t* sub_out, int32_t* i_out,
                   int32_t* j_out, int64_t* n_out) {
    if (!h || capacity < 0) return SSCF_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.last_sched_kind == 0) return SSCF_ERR_STATE;
    std::vector<int> pn(c.n_gnb), lvl((size_t)c.n_gnb * (kMaxSub + 1));
    std::vector<uint16_t> ij((size_t)c.n_gnb * kOrthoCap);
    CKA(cudaStreamSynchronize(c.stream));
    CKA(cudaMemcpy(pn.data(), c.d_pr_n, pn.size() * 4, cudaMemcpyDeviceToHost));
    CKA(cudaMemcpy(lvl.data(), c.d_pr_lvl, lvl.size() * 4, cudaMemcpyDeviceToHost));
    CKA(cudaMemcpy(ij.data(), c.d_pr_ij, ij.size() * 2, cudaMemcpyDeviceToHost));
    const bool rot = c.last_sched_kind == 1;
    const std::vector<int>& cptr = rot ? c.h_colour_ptr : c.h_ocolour_ptr;
    const std::vector<int>& cblk = rot ? c.h_colour_blk : c.h_ocolour_blk;
    const int w = c.last_sched_kind == 2 ? c.last_ortho_which : 0;
    int64_t k = 0;
    for (int col = 0; col < c.n_colours; ++col)
        for (int jb = cptr[col]; jb < cptr[col + 1]; ++jb) {
            const int e = cblk[jb];
            const int A = c.h_gnb_row[e], B = c.h_gnb_col[e];
            const int noA = 4 * c.h_group_nmol[A], noB = 4 * c.h_group_nmol[B];
            for (int sub = 0; sub < kMaxSub; ++sub)
                for (int q = lvl[(size_t)e * (kMaxSub + 1) + sub]; q < lvl[(size_t)e * (kMaxSub + 1) + sub + 1]; ++q) {
                    const unsigned v = ij[(size_t)e * kOrthoCap + q];
                    const int il = v & 255, jl = v >> 8;
                    int gi, gj;
                    if (rot) {
                        gi = c.h_group_occ0[A] + il;
                        gj = c.h_group_virt0[B] + jl;
                    } else {
                        gi = il < noA ? c.h_group_occ0[A] + il : c.h_group_virt0[A] + (il - noA);
                        gj = jl < noB ? c.h_group_occ0[B] + jl : c.h_group_virt0[B] + (jl - noB);
                        (void)w;
                    }
                    if (k < capacity) {
                        if (colour_out) colour_out[k] = col;
                        if (sub_out) sub_out[k] = sub;
                        if (i_out) i_out[k] = gi;
                        if (j_out) j_out[k] = gj;
                    }
                    ++k;
                }
        }
    if (n_out) *n_out = k;
    return SSCF_OK;
}

}  // extern "C"
