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
