// Adjoint of the SCC energy at the current (converged) MOs: forces and the
// gradients with respect to the eight Slater-Koster prefactors.
//
//   dE = sum P * dH0 + sum (P (Q_a + Q_b) / 2 - W) * dS + dq^T dgamma dq / 2,
//   W  = P H P / 2 = 2 C_o F_oo C_o^T,   F_oo = C_o^T H C_o,
//
// the first-order change of E = sum P H0 + dq^T gamma dq / 2 (Eq. H_dftb,
// Eq. pop) under the orthonormality constraint C^T S C = I with F_ov = 0.
// F_oo is formed on the occupied blocks of neighbouring groups (the same
// tile-pair transform as C^T S C), Z = C_o F_oo row by row, then P_mn and
// W_mn on the molecule-pair pattern are contracted with the analytic
// derivatives of the Slater-Koster blocks.
#include <math.h>

#include "sscf_internal.h"

namespace sscf {

namespace {

template <typename T> struct AccA;
template <> struct AccA<double> { using type = double; };
template <> struct AccA<float> { using type = float; };

// group-graph entry (g1, g2) with g1 <= g2, or -1
__device__ __forceinline__ int gnb_entry(const int* __restrict__ gnb_ptr, const int* __restrict__ gnb_col, int g1,
                                         int g2) {
    int lo = gnb_ptr[g1], hi = gnb_ptr[g1 + 1] - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = gnb_col[mid];
        if (v == g2) return mid;
        if (v < g2) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// F_oo[tB, tA] element (i, j) address inside the occupied tile-pair storage
// (blocks A <= B, inside one group a <= b); transposed when stored the other way
struct FRef {
    int tp;
    bool transposed;
};

__device__ __forceinline__ FRef f_ref(const int* gnb_ptr, const int* gnb_col, const int* self_blk,
                                      const int* blk_tp, const int* group_ot0, int gB, int tB, int gA, int tA) {
    const int posB = tB - group_ot0[gB], posA = tA - group_ot0[gA];
    FRef f{-1, false};
    if (gB < gA) {
        const int e = gnb_entry(gnb_ptr, gnb_col, gB, gA);
        if (e >= 0) f.tp = blk_tp[e * 9 + posB * 3 + posA];
    } else if (gB > gA) {
        const int e = gnb_entry(gnb_ptr, gnb_col, gA, gB);
        if (e >= 0) {
            f.tp = blk_tp[e * 9 + posA * 3 + posB];
            f.transposed = true;
        }
    } else {
        const int e = self_blk[gA];
        if (posB <= posA) {
            f.tp = blk_tp[e * 9 + posB * 3 + posA];
        } else {
            f.tp = blk_tp[e * 9 + posA * 3 + posB];
            f.transposed = true;
        }
    }
    return f;
}

// Z = C_o F_oo, row-major like C. Row block r gets the occupied tiles of every
// group adjacent (or equal) to a group whose occupied tiles it holds; one warp
// per output tile sums C[r, tB] F_oo[tB, tA] over r's tiles tB of adjacent groups.
template <typename T>
__global__ void __launch_bounds__(256) k_zmul(int n_tiles, int n_occ_tiles, int n_groups, int cap,
                                              const int* __restrict__ c_nt, const int* __restrict__ c_tile,
                                              const T* __restrict__ c_val, const int* __restrict__ tile_group,
                                              const int* __restrict__ group_ot0, const int* __restrict__ group_not,
                                              const int* __restrict__ gnb_ptr, const int* __restrict__ gnb_col,
                                              const int* __restrict__ self_blk, const int* __restrict__ blk_tp,
                                              const T* __restrict__ F, int* __restrict__ z_nt,
                                              int* __restrict__ z_tile, T* __restrict__ z_val,
                                              unsigned* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int gw = (n_groups + 31) >> 5;
    unsigned* pres = (unsigned*)smraw;          // gw: groups with occupied tiles in row r
    unsigned* outg = pres + gw;                 // gw: groups of Z's tiles
    int* in_t = (int*)(outg + gw);              // cap: r's occupied tiles
    int* in_s = in_t + cap;                     // cap: their slots
    int* out_t = in_s + cap;                    // cap: Z's tiles
    __shared__ int part[256];
    __shared__ int s_nin, s_nout;
    const int r = blockIdx.x;
    for (int i = threadIdx.x; i < gw; i += blockDim.x) pres[i] = outg[i] = 0u;
    if (threadIdx.x == 0) s_nin = 0;
    __syncthreads();
    const int n0 = c_nt[r];
    if (threadIdx.x == 0) {
        int k = 0;
        for (int s = 0; s < n0; ++s) {
            const int t = c_tile[(size_t)r * cap + s];
            if (t >= n_occ_tiles) break;
            in_t[k] = t;
            in_s[k] = s;
            ++k;
        }
        s_nin = k;
    }
    __syncthreads();
    const int nin = s_nin;
    for (int k = threadIdx.x; k < nin; k += blockDim.x) {
        const int g = tile_group[in_t[k]];
        atomicOr(&pres[g >> 5], 1u << (g & 31));
    }
    __syncthreads();
    for (int g = threadIdx.x; g < n_groups; g += blockDim.x) {
        if (!((pres[g >> 5] >> (g & 31)) & 1)) continue;
        for (int e = gnb_ptr[g]; e < gnb_ptr[g + 1]; ++e) {
            const int B = gnb_col[e];
            atomicOr(&outg[B >> 5], 1u << (B & 31));
        }
    }
    __syncthreads();
    // sorted output tile list (occupied tiles, group order)
    const int per = (n_groups + blockDim.x - 1) / blockDim.x;
    const int g0 = threadIdx.x * per, g1 = min(n_groups, g0 + per);
    int cnt = 0;
    for (int g = g0; g < g1; ++g)
        if ((outg[g >> 5] >> (g & 31)) & 1) cnt += group_not[g];
    part[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
        s_nout = run;
    }
    __syncthreads();
    const int nout = s_nout;
    if (nout > cap) {
        if (threadIdx.x == 0) {
            atomicOr(err, kErrCapacity);
            z_nt[r] = 0;
        }
        return;
    }
    int pos = part[threadIdx.x];
    for (int g = g0; g < g1; ++g)
        if ((outg[g >> 5] >> (g & 31)) & 1)
            for (int i = 0; i < group_not[g]; ++i) out_t[pos++] = group_ot0[g] + i;
    __syncthreads();
    if (threadIdx.x == 0) z_nt[r] = nout;
    for (int s = threadIdx.x; s < nout; s += blockDim.x) z_tile[(size_t)r * cap + s] = out_t[s];
    using A = typename AccA<T>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int j = lane & 15, kh = lane >> 4;
    for (int s = warp; s < nout; s += nwarps) {
        const int tA = out_t[s];
        const int gA = tile_group[tA];
        A acc[3] = {0, 0, 0};
        for (int k = 0; k < nin; ++k) {
            const int tB = in_t[k];
            const int gB = tile_group[tB];
            const FRef f = f_ref(gnb_ptr, gnb_col, self_blk, blk_tp, group_ot0, gB, tB, gA, tA);
            if (f.tp < 0) continue;
            const T* cv = c_val + ((size_t)r * cap + in_s[k]) * kTileVals;
            const T* fv = F + (size_t)f.tp * 256;
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const A fij = (A)(f.transposed ? fv[j * 16 + i] : fv[i * 16 + j]);
                acc[0] += (A)cv[(kh)*16 + i] * fij;
                acc[1] += (A)cv[(kh + 2) * 16 + i] * fij;
                acc[2] += (A)cv[(kh + 4) * 16 + i] * fij;
            }
        }
        T* zv = z_val + ((size_t)r * cap + s) * kTileVals;
        zv[(kh)*16 + j] = (T)acc[0];
        zv[(kh + 2) * 16 + j] = (T)acc[1];
        zv[(kh + 4) * 16 + j] = (T)acc[2];
    }
}

struct SKd {
    double V0[4], S0[4];
    double r_decay, rc2;
};

__device__ __forceinline__ double dist2_rn(const double* a, const double* b) {
    double dx = __dsub_rn(b[0], a[0]);
    double dy = __dsub_rn(b[1], a[1]);
    double dz = __dsub_rn(b[2], a[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ int ao_off(int k) { return k == 0 ? 0 : 3 + k; }

// Contribution of the ordered atom pair (a in m, b in n) to dE: the force on
// atom a (-2 g, g = sum P dH/dR + GS dS/dR, R = x_b - x_a; the pair (b, a)
// gives the same on a) and the parameter partials sum P H0^(k) and GS S^(k).
__device__ void pair_terms(const SKd& P, const double* xa, const double* xb, int na, int nb, int oa, int ob,
                           const double* Pm, const double* GS, double* fa, double* dpar) {
    double d2 = dist2_rn(xa, xb);
    if (!(d2 <= P.rc2)) return;
    const double r = sqrt(d2);
    double e[3], R[3];
    for (int d = 0; d < 3; ++d) {
        R[d] = xb[d] - xa[d];
        e[d] = R[d] / r;
    }
    const double decay = exp(-r / P.r_decay);
    for (int tab = 0; tab < 2; ++tab) {
        const double* V0 = tab == 0 ? P.V0 : P.S0;
        const double* Wt = tab == 0 ? Pm : GS;
        double V[4], dV[4];
        for (int q = 0; q < 4; ++q) {
            V[q] = V0[q] * decay;
            dV[q] = -V[q] / P.r_decay;
        }
        double g[3] = {0, 0, 0};
        double par[4] = {0, 0, 0, 0};
        for (int i = 0; i < na; ++i)
            for (int jj = 0; jj < nb; ++jj) {
                const double w = Wt[(oa + i) * 6 + ob + jj];
                if (w == 0.0) continue;
                for (int k = 0; k < 3; ++k) {
                    double v;
                    if (i == 0 && jj == 0) {
                        v = dV[0] * e[k];
                    } else if (i == 0 || jj == 0) {
                        const int c = i == 0 ? jj - 1 : i - 1;
                        const double dec = ((c == k ? 1.0 : 0.0) - e[c] * e[k]) / r;
                        v = dec * V[1] + e[c] * dV[1] * e[k];
                        if (jj == 0) v = -v;
                    } else {
                        const int ci = i - 1, cj = jj - 1;
                        const double dei = ((ci == k ? 1.0 : 0.0) - e[ci] * e[k]) / r;
                        const double dej = ((cj == k ? 1.0 : 0.0) - e[cj] * e[k]) / r;
                        v = (dei * e[cj] + e[ci] * dej) * (V[2] - V[3]) + e[ci] * e[cj] * (dV[2] - dV[3]) * e[k] +
                            (ci == cj ? dV[3] * e[k] : 0.0);
                    }
                    g[k] += w * v;
                }
                // parameter partials: the block is linear in the prefactors
                if (i == 0 && jj == 0) {
                    par[0] += w * decay;
                } else if (i == 0 || jj == 0) {
                    const int c = i == 0 ? jj - 1 : i - 1;
                    par[1] += w * (jj == 0 ? -e[c] : e[c]) * decay;
                } else {
                    const int ci = i - 1, cj = jj - 1;
                    par[2] += w * e[ci] * e[cj] * decay;
                    par[3] += w * ((ci == cj ? 1.0 : 0.0) - e[ci] * e[cj]) * decay;
                }
            }
        for (int k = 0; k < 3; ++k) fa[k] += -2.0 * g[k];
        for (int q = 0; q < 4; ++q) dpar[tab * 4 + q] += par[q];
    }
}

// One CTA per row block m, one warp per pattern neighbour n: P_mn and
// W_mn = 2 sum_t C[m,t] Z[n,t]^T on the tiles both rows hold, then the pair
// terms of the 9 atom pairs; per-molecule partials summed in neighbour order.
constexpr int kGradWarps = 8;
template <typename T>
__global__ void __launch_bounds__(kGradWarps * 32)
k_grad_blocks(int n_occ_tiles, int map_n, const int* __restrict__ mol_ot0, int cap, const int* __restrict__ c_nt,
              const int* __restrict__ c_tile,
              const T* __restrict__ c_val, const int* __restrict__ z_nt, const int* __restrict__ z_tile,
              const T* __restrict__ z_val, const int* __restrict__ mp_ptr, const int* __restrict__ mp_col,
              const double* __restrict__ xyz, const double* __restrict__ Q, SKd P, double* __restrict__ gmol,
              double* __restrict__ pmol) {
    extern __shared__ int smap[];   // map_n: slot in C row m of each occupied tile of m's cluster, or -1
    __shared__ double part[kGradWarps][17];
    const int m = blockIdx.x;
    const int t0 = mol_ot0[m];
    for (int i = threadIdx.x; i < map_n; i += blockDim.x) smap[i] = -1;
    __syncthreads();
    const int ntm = c_nt[m];
    for (int s = threadIdx.x; s < ntm; s += blockDim.x) {
        const int t = c_tile[(size_t)m * cap + s];
        if (t < n_occ_tiles) smap[t - t0] = s;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e0 = mp_ptr[m], ne = mp_ptr[m + 1] - e0;
    const int col = lane & 15, half = lane >> 4;
    using A = typename AccA<T>::type;
    double wsum[17];
    for (int u = 0; u < 17; ++u) wsum[u] = 0.0;
    for (int w = warp; w < ne; w += kGradWarps) {
        const int n = mp_col[e0 + w];
        double accP[36], accW[36];
        for (int u = 0; u < 36; ++u) accP[u] = accW[u] = 0.0;
        const int ntn = c_nt[n];
        for (int s = half; s < ntn; s += 2) {
            const int t = c_tile[(size_t)n * cap + s];
            if (t >= n_occ_tiles) break;
            const int sm_ = smap[t - t0];
            if (sm_ < 0) continue;
            const T* cm = c_val + ((size_t)m * cap + sm_) * kTileVals + col;
            const T* cn = c_val + ((size_t)n * cap + s) * kTileVals + col;
            A a6[6], b6[6];
            for (int k = 0; k < 6; ++k) {
                a6[k] = (A)cm[k * kTileW];
                b6[k] = (A)cn[k * kTileW];
            }
            for (int k = 0; k < 6; ++k)
                for (int l = 0; l < 6; ++l) accP[k * 6 + l] += (double)(a6[k] * b6[l]);
        }
        const int nzn = z_nt[n];
        for (int s = half; s < nzn; s += 2) {
            const int t = z_tile[(size_t)n * cap + s];
            const int sm_ = smap[t - t0];
            if (sm_ < 0) continue;
            const T* cm = c_val + ((size_t)m * cap + sm_) * kTileVals + col;
            const T* zn = z_val + ((size_t)n * cap + s) * kTileVals + col;
            A a6[6], b6[6];
            for (int k = 0; k < 6; ++k) {
                a6[k] = (A)cm[k * kTileW];
                b6[k] = (A)zn[k * kTileW];
            }
            for (int k = 0; k < 6; ++k)
                for (int l = 0; l < 6; ++l) accW[k * 6 + l] += (double)(a6[k] * b6[l]);
        }
        for (int u = 0; u < 36; ++u) {
            for (int off = 16; off > 0; off >>= 1) {
                accP[u] += __shfl_xor_sync(0xffffffffu, accP[u], off);
                accW[u] += __shfl_xor_sync(0xffffffffu, accW[u], off);
            }
        }
        // lanes 0..8: atom pair (a in m, b in n)
        double fa[3] = {0, 0, 0}, dp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (lane < 9) {
            const int ia = lane / 3, ib = lane % 3;
            const int a = 3 * m + ia, b = 3 * n + ib;
            if (a != b) {
                double Pm[36], GS[36];
                for (int u = 0; u < 36; ++u) {
                    const int k = u / 6, l = u % 6;
                    const int at_k = 3 * m + (k < 4 ? 0 : k - 3), at_l = 3 * n + (l < 4 ? 0 : l - 3);
                    Pm[u] = 2.0 * accP[u];
                    GS[u] = 0.5 * Pm[u] * (Q[at_k] + Q[at_l]) - 2.0 * accW[u];
                }
                pair_terms(P, xyz + 3 * a, xyz + 3 * b, ia == 0 ? 4 : 1, ib == 0 ? 4 : 1, ao_off(ia), ao_off(ib), Pm,
                           GS, fa, dp);
            }
        }
        // gather the 9 pair results into lane 0 (fixed order)
        for (int src = 0; src < 9; ++src) {
            const double f0 = __shfl_sync(0xffffffffu, fa[0], src), f1 = __shfl_sync(0xffffffffu, fa[1], src),
                         f2 = __shfl_sync(0xffffffffu, fa[2], src);
            double pp[8];
            for (int q = 0; q < 8; ++q) pp[q] = __shfl_sync(0xffffffffu, dp[q], src);
            const int ia = src / 3;
            wsum[ia * 3 + 0] += f0;
            wsum[ia * 3 + 1] += f1;
            wsum[ia * 3 + 2] += f2;
            for (int q = 0; q < 8; ++q) wsum[9 + q] += pp[q];
        }
    }
    if (lane == 0)
        for (int u = 0; u < 17; ++u) part[warp][u] = wsum[u];
    __syncthreads();
    if (threadIdx.x < 17) {
        double s = 0.0;
        for (int w = 0; w < kGradWarps; ++w) s += part[w][threadIdx.x];
        if (threadIdx.x < 9)
            gmol[(size_t)m * 9 + threadIdx.x] = s;
        else
            pmol[(size_t)m * 8 + threadIdx.x - 9] = s;
    }
}

// dE/dx_a of dq^T gamma dq / 2: -dq_a sum_b dq_b gamma_ab^3 (x_a - x_b)
__global__ void k_gamma_force(int n, const double* __restrict__ xyz, const int* __restrict__ species,
                              const int* __restrict__ atom_lo, const int* __restrict__ atom_hi,
                              const double* __restrict__ dq, double invU0, double invU1, double* __restrict__ out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int b_lo = atom_lo[a], b_hi = atom_hi[a];   // gamma couples atoms of one cluster only
    const double xa = xyz[3 * a], ya = xyz[3 * a + 1], za = xyz[3 * a + 2];
    const double ia = species[a] == 0 ? invU0 : invU1;
    double f[3] = {0, 0, 0};
    for (int b = b_lo; b < b_hi; ++b) {
        if (b == a) continue;
        const double dx = xa - xyz[3 * b], dy = ya - xyz[3 * b + 1], dz = za - xyz[3 * b + 2];
        const double h = 0.5 * (ia + (species[b] == 0 ? invU0 : invU1));
        const double g = 1.0 / sqrt(dx * dx + dy * dy + dz * dz + h * h);
        const double w = dq[b] * g * g * g;
        f[0] += w * dx;
        f[1] += w * dy;
        f[2] += w * dz;
    }
    for (int d = 0; d < 3; ++d) out[3 * a + d] = -dq[a] * f[d];
}

__global__ void k_grad_finish(int n_mol, const double* __restrict__ gmol, const double* __restrict__ pmol,
                              double* __restrict__ grad, double* __restrict__ dpar) {
    for (int i = threadIdx.x; i < 9 * n_mol; i += blockDim.x) grad[i] += gmol[i];
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int m = 0; m < n_mol; ++m) s += pmol[(size_t)m * 8 + threadIdx.x];
        dpar[threadIdx.x] = s;
    }
}

}  // namespace

template <typename T>
static cudaError_t adjoint_t(Ctx* c, double* d_grad, double* d_par, double* d_gmol, double* d_pmol) {
    const int in = c->cur, zb = 1 - c->cur;
    const int gw = (c->n_groups + 31) / 32;
    const size_t smem_z = (size_t)2 * gw * 4 + (size_t)3 * c->cap * 4;
    if (smem_z > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_zmul<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_z);
    if (e != cudaSuccess) return e;
    k_zmul<T><<<c->n_mol, 256, smem_z, c->stream>>>(
        c->n_tiles, c->n_occ_tiles, c->n_groups, c->cap, c->d_c_nt[in], c->d_c_tile[in], (const T*)c->d_c_val[in],
        c->d_tile_group, c->d_group_ot0, c->d_group_not, c->d_gnb_ptr, c->d_gnb_col, c->d_self_blk,
        c->d_ort_blk_tp[1], (const T*)c->d_sig, c->d_c_nt[zb], c->d_c_tile[zb], (T*)c->d_c_val[zb], &c->d_sc->err);
    SKd P;
    for (int i = 0; i < 4; ++i) {
        P.V0[i] = c->prm.V0[i];
        P.S0[i] = c->prm.S0[i];
    }
    P.r_decay = c->prm.r_decay;
    P.rc2 = c->prm.r_cut * c->prm.r_cut;
    const size_t smem_g = (size_t)c->max_cl_otiles * 4;
    e = cudaFuncSetAttribute(k_grad_blocks<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g);
    if (e != cudaSuccess) return e;
    k_grad_blocks<T><<<c->n_mol, kGradWarps * 32, smem_g, c->stream>>>(
        c->n_occ_tiles, c->max_cl_otiles, c->d_mol_ot0, c->cap, c->d_c_nt[in], c->d_c_tile[in], (const T*)c->d_c_val[in], c->d_c_nt[zb],
        c->d_c_tile[zb], (const T*)c->d_c_val[zb], c->d_mp_ptr, c->d_mp_col, c->d_xyz, c->d_Q, P, d_gmol, d_pmol);
    k_gamma_force<<<(c->n_atoms + 127) / 128, 128, 0, c->stream>>>(c->n_atoms, c->d_xyz, c->d_species, c->d_atom_lo,
                                                                  c->d_atom_hi, c->d_dq,
                                                                  1.0 / c->prm.U[0], 1.0 / c->prm.U[1], d_grad);
    k_grad_finish<<<1, 1024, 0, c->stream>>>(c->n_mol, d_gmol, d_pmol, d_grad, d_par);
    c->n_launch += 4;
    return cudaGetLastError();
}

cudaError_t launch_adjoint(Ctx* c, double* d_grad, double* d_par, double* d_gmol, double* d_pmol) {
    return c->prec == SSCF_FP64 ? adjoint_t<double>(c, d_grad, d_par, d_gmol, d_pmol)
                                : adjoint_t<float>(c, d_grad, d_par, d_gmol, d_pmol);
}

}  // namespace sscf
