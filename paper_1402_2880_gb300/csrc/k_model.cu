// Model kernels: Slater-Koster H0 / S blocks, the SCC shift Q = gamma dq,
// the DFTB Hamiltonian of Eq. (H_dftb2) and the per-molecule initial guess.
#include <math.h>

#include "sscf_internal.h"

namespace sscf {

namespace {

struct SK {
    double onsite[3];
    double V0[4], S0[4];
    double r_decay, rc2;
    double U[2];
};

__device__ __forceinline__ double dist2_rn(const double* a, const double* b) {
    double dx = __dsub_rn(b[0], a[0]);
    double dy = __dsub_rn(b[1], a[1]);
    double dz = __dsub_rn(b[2], a[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// AO offset inside a water molecule of atom k (0 = O: AOs 0..3, 1 = H1: 4, 2 = H2: 5)
__device__ __forceinline__ int ao_off(int k) { return k == 0 ? 0 : 3 + k; }

// One thread per molecule-pair block (m, n): the 6x6 blocks of H0 and S.
// Two-centre elements follow the Slater-Koster direction-cosine rules with
// V(r) = V0 exp(-r / r_decay) for every pair with r <= r_cut; the diagonal
// block carries the on-site energies and S = 1 on the atom diagonals.
__global__ void k_sk_blocks(int n_mp, const int* __restrict__ mp_row, const int* __restrict__ mp_col,
                            const double* __restrict__ xyz, SK P, double* __restrict__ H0b,
                            double* __restrict__ Sb) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_mp) return;
    const int m = mp_row[k], n = mp_col[k];
    double h[36], s[36];
#pragma unroll
    for (int i = 0; i < 36; ++i) h[i] = s[i] = 0.0;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            const int ia = 3 * m + a, ib = 3 * n + b;
            const int oa = ao_off(a), ob = ao_off(b);
            const int na = a == 0 ? 4 : 1, nb = b == 0 ? 4 : 1;
            if (ia == ib) {
                for (int i = 0; i < na; ++i) {
                    double e = a == 0 ? (i == 0 ? P.onsite[0] : P.onsite[1]) : P.onsite[2];
                    h[(oa + i) * 6 + oa + i] = e;
                    s[(oa + i) * 6 + oa + i] = 1.0;
                }
                continue;
            }
            const double* xa = xyz + 3 * ia;
            const double* xb = xyz + 3 * ib;
            double d2 = dist2_rn(xa, xb);
            if (!(d2 <= P.rc2)) continue;
            double r = sqrt(d2);
            double e3[3];
            for (int d = 0; d < 3; ++d) e3[d] = __ddiv_rn(__dsub_rn(xb[d], xa[d]), r);
            double decay = exp(-__ddiv_rn(r, P.r_decay));
            for (int tab = 0; tab < 2; ++tab) {
                const double* V = tab == 0 ? P.V0 : P.S0;
                double* out = tab == 0 ? h : s;
                double Vss = __dmul_rn(V[0], decay), Vsp = __dmul_rn(V[1], decay);
                double Vpps = __dmul_rn(V[2], decay), Vppp = __dmul_rn(V[3], decay);
                for (int i = 0; i < na; ++i)
                    for (int j = 0; j < nb; ++j) {
                        double v;
                        if (i == 0 && j == 0) {
                            v = Vss;
                        } else if (i == 0) {
                            v = __dmul_rn(e3[j - 1], Vsp);
                        } else if (j == 0) {
                            v = __dmul_rn(-e3[i - 1], Vsp);
                        } else {
                            v = __dmul_rn(__dmul_rn(e3[i - 1], e3[j - 1]), __dsub_rn(Vpps, Vppp));
                            if (i == j) v = __dadd_rn(v, Vppp);
                        }
                        out[(oa + i) * 6 + ob + j] = v;
                    }
            }
        }
    }
    for (int i = 0; i < 36; ++i) {
        H0b[(size_t)k * 36 + i] = h[i];
        Sb[(size_t)k * 36 + i] = s[i];
    }
}

// Q_a = sum_b gamma_ab dq_b over all atom pairs (unscreened, Section
// "Specific implementation for DFTB"), gamma_ab = 1/sqrt(r^2 + a^2),
// a = (1/U_a + 1/U_b)/2. One thread per atom a, atoms b staged in smem.
// P = double: every pair term in FP64. P = float (mixed precision): pair
// terms in FP32, summed in FP32 over one smem tile of 256 atoms, tile sums
// accumulated in FP64.
constexpr int kGammaTile = 256;
template <typename P>
__global__ void k_gamma(int n, const double* __restrict__ xyz, const int* __restrict__ species,
                        const int* __restrict__ atom_lo, const int* __restrict__ atom_hi,
                        const double* __restrict__ dq, double invU0, double invU1, double* __restrict__ Q) {
    __shared__ P sx[kGammaTile * 3];
    __shared__ P sq[kGammaTile];
    __shared__ P si[kGammaTile];
    __shared__ int s_lo, s_hi;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double xa_d[3] = {0, 0, 0}, ia_d = invU0;
    int lo = 1 << 30, hi = -1;   // gamma couples atoms of one cluster only
    if (a < n) {
        xa_d[0] = xyz[3 * a];
        xa_d[1] = xyz[3 * a + 1];
        xa_d[2] = xyz[3 * a + 2];
        ia_d = species[a] == 0 ? invU0 : invU1;
        lo = atom_lo[a];
        hi = atom_hi[a];
    }
    if (threadIdx.x == 0) {
        s_lo = 1 << 30;
        s_hi = -1;
    }
    __syncthreads();
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
    __syncthreads();
    const P xa[3] = {(P)xa_d[0], (P)xa_d[1], (P)xa_d[2]};
    const P ia = (P)ia_d;
    double acc = 0.0;
    const int blo = s_lo, bhi = s_hi;
    for (int b0 = blo; b0 < bhi; b0 += kGammaTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kGammaTile; t += blockDim.x) {
            int b = b0 + t;
            if (b < bhi) {
                sx[3 * t] = (P)xyz[3 * b];
                sx[3 * t + 1] = (P)xyz[3 * b + 1];
                sx[3 * t + 2] = (P)xyz[3 * b + 2];
                sq[t] = (P)dq[b];
                si[t] = (P)(species[b] == 0 ? invU0 : invU1);
            } else {
                sx[3 * t] = sx[3 * t + 1] = sx[3 * t + 2] = (P)0;
                sq[t] = (P)0;
                si[t] = (P)invU0;
            }
        }
        __syncthreads();
        const int nb = min(kGammaTile, bhi - b0);
        P part = 0;
        const int t_lo = max(0, lo - b0), t_hi = min(nb, hi - b0);
        for (int t = t_lo; t < t_hi; ++t) {
            const P dx = sx[3 * t] - xa[0], dy = sx[3 * t + 1] - xa[1], dz = sx[3 * t + 2] - xa[2];
            const P d2 = dx * dx + dy * dy + dz * dz;
            const P h = (P)0.5 * (ia + si[t]);
            part += sq[t] / sqrt(d2 + h * h);
        }
        acc += (double)part;
    }
    if (a < n) Q[a] = acc;
}

// H = H0 + 1/2 S (Q_a + Q_b) on every molecule-pair block (Eq. H_dftb2);
// off-diagonal |H| < eps set to zero. Also stores S in the storage type.
template <typename T>
__global__ void k_build_h(int n_mp, const int* __restrict__ mp_row, const int* __restrict__ mp_col,
                          const double* __restrict__ H0b, const double* __restrict__ Sb,
                          const double* __restrict__ Q, double eps, T* __restrict__ Hb, T* __restrict__ Sbt) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_mp * 36) return;
    const int k = idx / 36, e = idx % 36;
    const int m = mp_row[k], n = mp_col[k];
    const int i = e / 6, j = e % 6;
    const int ai = 3 * m + (i < 4 ? 0 : i - 3);
    const int bj = 3 * n + (j < 4 ? 0 : j - 3);
    double s = Sb[idx];
    double h = __dadd_rn(H0b[idx], __dmul_rn(__dmul_rn(0.5, s), __dadd_rn(Q[ai], Q[bj])));
    bool diag = (m == n) && (i == j);
    if (!diag && fabs(h) < eps) h = 0.0;
    Hb[idx] = (T)h;
    Sbt[idx] = (T)s;
}

// ---- per-molecule generalised eigensolve (step II) --------------------------
// Cholesky S = L L^T, A = L^-1 H L^-T, cyclic Jacobi on A, x = L^-T v.
__device__ bool small_geneig6(const double* Hm, const double* Sm, double* w, double* X) {
    double L[36];
    for (int i = 0; i < 36; ++i) L[i] = 0.0;
    for (int j = 0; j < 6; ++j) {
        double d = Sm[j * 6 + j];
        for (int k = 0; k < j; ++k) d -= L[j * 6 + k] * L[j * 6 + k];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        L[j * 6 + j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double v = Sm[i * 6 + j];
            for (int k = 0; k < j; ++k) v -= L[i * 6 + k] * L[j * 6 + k];
            L[i * 6 + j] = v / d;
        }
    }
    // Linv (lower triangular inverse)
    double Li[36];
    for (int i = 0; i < 36; ++i) Li[i] = 0.0;
    for (int j = 0; j < 6; ++j) {
        Li[j * 6 + j] = 1.0 / L[j * 6 + j];
        for (int i = j + 1; i < 6; ++i) {
            double v = 0.0;
            for (int k = j; k < i; ++k) v -= L[i * 6 + k] * Li[k * 6 + j];
            Li[i * 6 + j] = v / L[i * 6 + i];
        }
    }
    double A[36], T1[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0.0;
            for (int k = 0; k < 6; ++k) v += Li[i * 6 + k] * Hm[k * 6 + j];
            T1[i * 6 + j] = v;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0.0;
            for (int k = 0; k < 6; ++k) v += T1[i * 6 + k] * Li[j * 6 + k];
            A[i * 6 + j] = v;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < i; ++j) A[i * 6 + j] = A[j * 6 + i] = 0.5 * (A[i * 6 + j] + A[j * 6 + i]);
    double V[36];
    for (int i = 0; i < 36; ++i) V[i] = (i % 7 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                tot += A[i * 6 + j] * A[i * 6 + j];
                if (i != j) off += A[i * 6 + j] * A[i * 6 + j];
            }
        if (off <= 1e-34 * tot) break;
        for (int p = 0; p < 5; ++p)
            for (int q = p + 1; q < 6; ++q) {
                double apq = A[p * 6 + q];
                if (apq == 0.0) continue;
                double theta = (A[q * 6 + q] - A[p * 6 + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 6; ++k) {
                    double akp = A[k * 6 + p], akq = A[k * 6 + q];
                    A[k * 6 + p] = cs * akp - sn * akq;
                    A[k * 6 + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 6; ++k) {
                    double apk = A[p * 6 + k], aqk = A[q * 6 + k];
                    A[p * 6 + k] = cs * apk - sn * aqk;
                    A[q * 6 + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 6; ++k) {
                    double vkp = V[k * 6 + p], vkq = V[k * 6 + q];
                    V[k * 6 + p] = cs * vkp - sn * vkq;
                    V[k * 6 + q] = sn * vkp + cs * vkq;
                }
            }
    }
    // sort ascending
    int ord[6];
    for (int i = 0; i < 6; ++i) ord[i] = i;
    for (int i = 1; i < 6; ++i)
        for (int j = i; j > 0 && A[ord[j] * 7] < A[ord[j - 1] * 7]; --j) {
            int t = ord[j];
            ord[j] = ord[j - 1];
            ord[j - 1] = t;
        }
    for (int n = 0; n < 6; ++n) {
        const int src = ord[n];
        w[n] = A[src * 7];
        // x = L^-T v
        double x[6];
        for (int i = 0; i < 6; ++i) {
            double v = 0.0;
            for (int k = 0; k < 6; ++k) v += Li[k * 6 + i] * V[k * 6 + src];
            x[i] = v;
        }
        double amax = 0.0;
        for (int i = 0; i < 6; ++i) amax = fmax(amax, fabs(x[i]));
        int kk = 0;
        for (int i = 0; i < 6; ++i)
            if (fabs(x[i]) >= amax * (1.0 - 1e-9)) {
                kk = i;
                break;
            }
        double sg = x[kk] > 0 ? 1.0 : -1.0;
        for (int i = 0; i < 6; ++i) X[i * 6 + n] = sg * x[i];
    }
    return true;
}

// One thread per molecule: the molecule's guess MOs become columns of its
// group's tiles; row block m gets exactly its occupied tile and its virtual
// tile (other columns zero).
template <typename T>
__global__ void k_guess(int n_mol, const int* __restrict__ mp_ptr, const int* __restrict__ mp_col,
                        const double* __restrict__ H0b, const double* __restrict__ Sb,
                        const int* __restrict__ mol_group, const int* __restrict__ mol_local,
                        const int* __restrict__ group_ot0, const int* __restrict__ group_vt0, int cap,
                        int* __restrict__ c_nt, int* __restrict__ c_tile, T* __restrict__ c_val,
                        unsigned* __restrict__ err) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mol) return;
    int kd = -1;
    for (int k = mp_ptr[m]; k < mp_ptr[m + 1]; ++k)
        if (mp_col[k] == m) kd = k;
    double w[6], X[36];
    bool ok = kd >= 0 && small_geneig6(H0b + (size_t)kd * 36, Sb + (size_t)kd * 36, w, X);
    if (!ok) {
        atomicOr(err, kErrGuess);
        c_nt[m] = 0;
        return;
    }
    const int g = mol_group[m], loc = mol_local[m];
    const int to = group_ot0[g] + (4 * loc) / kTileW, co = (4 * loc) % kTileW;
    const int tv = group_vt0[g] + (2 * loc) / kTileW, cv = (2 * loc) % kTileW;
    c_nt[m] = 2;
    c_tile[(size_t)m * cap + 0] = to;
    c_tile[(size_t)m * cap + 1] = tv;
    T* vo = c_val + (size_t)m * cap * kTileVals;
    T* vv = vo + kTileVals;
    for (int i = 0; i < kTileVals; ++i) {
        vo[i] = (T)0;
        vv[i] = (T)0;
    }
    for (int r = 0; r < 6; ++r) {
        for (int n = 0; n < 4; ++n) vo[r * kTileW + co + n] = (T)X[r * 6 + n];
        for (int n = 0; n < 2; ++n) vv[r * kTileW + cv + n] = (T)X[r * 6 + 4 + n];
    }
}

SK make_sk(const Ctx* c) {
    SK P;
    for (int i = 0; i < 3; ++i) P.onsite[i] = c->prm.onsite[i];
    for (int i = 0; i < 4; ++i) {
        P.V0[i] = c->prm.V0[i];
        P.S0[i] = c->prm.S0[i];
    }
    P.r_decay = c->prm.r_decay;
    P.rc2 = c->prm.r_cut * c->prm.r_cut;
    P.U[0] = c->prm.U[0];
    P.U[1] = c->prm.U[1];
    return P;
}

}  // namespace

cudaError_t launch_sk_blocks(Ctx* c) {
    c->n_launch += 1;
    const int th = 128;
    k_sk_blocks<<<(c->n_mp + th - 1) / th, th, 0, c->stream>>>(c->n_mp, c->d_mp_row, c->d_mp_col, c->d_xyz,
                                                              make_sk(c), c->d_H0b, c->d_Sb);
    return cudaGetLastError();
}

cudaError_t launch_gamma(Ctx* c, const double* dq, double* Q) {
    c->n_launch += 1;
    const int th = 256;
    if (c->prec == SSCF_FP64)
        k_gamma<double><<<(c->n_atoms + th - 1) / th, th, 0, c->stream>>>(c->n_atoms, c->d_xyz, c->d_species,
                                                                          c->d_atom_lo, c->d_atom_hi, dq,
                                                                          1.0 / c->prm.U[0], 1.0 / c->prm.U[1], Q);
    else
        k_gamma<float><<<(c->n_atoms + th - 1) / th, th, 0, c->stream>>>(c->n_atoms, c->d_xyz, c->d_species,
                                                                         c->d_atom_lo, c->d_atom_hi, dq,
                                                                         1.0 / c->prm.U[0], 1.0 / c->prm.U[1], Q);
    return cudaGetLastError();
}

cudaError_t launch_build_h(Ctx* c, double eps_threshold) {
    c->n_launch += 1;
    const int th = 256;
    const int n = c->n_mp * 36;
    if (c->prec == SSCF_FP64)
        k_build_h<double><<<(n + th - 1) / th, th, 0, c->stream>>>(c->n_mp, c->d_mp_row, c->d_mp_col, c->d_H0b,
                                                                    c->d_Sb, c->d_Q_in, eps_threshold,
                                                                    (double*)c->d_Hb, (double*)c->d_Sbt);
    else
        k_build_h<float><<<(n + th - 1) / th, th, 0, c->stream>>>(c->n_mp, c->d_mp_row, c->d_mp_col, c->d_H0b,
                                                                   c->d_Sb, c->d_Q_in, eps_threshold,
                                                                   (float*)c->d_Hb, (float*)c->d_Sbt);
    return cudaGetLastError();
}

cudaError_t launch_guess(Ctx* c) {
    c->n_launch += 1;
    const int th = 64;
    c->cur = 0;
    if (c->prec == SSCF_FP64)
        k_guess<double><<<(c->n_mol + th - 1) / th, th, 0, c->stream>>>(
            c->n_mol, c->d_mp_ptr, c->d_mp_col, c->d_H0b, c->d_Sb, c->d_mol_group, c->d_mol_local,
            c->d_group_ot0, c->d_group_vt0, c->cap, c->d_c_nt[0], c->d_c_tile[0], (double*)c->d_c_val[0],
            &c->d_sc->err);
    else
        k_guess<float><<<(c->n_mol + th - 1) / th, th, 0, c->stream>>>(
            c->n_mol, c->d_mp_ptr, c->d_mp_col, c->d_H0b, c->d_Sb, c->d_mol_group, c->d_mol_local,
            c->d_group_ot0, c->d_group_vt0, c->cap, c->d_c_nt[0], c->d_c_tile[0], (float*)c->d_c_val[0],
            &c->d_sc->err);
    return cudaGetLastError();
}

}  // namespace sscf
