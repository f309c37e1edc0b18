// Charge update of one SCC iteration: dq = q - q0, Q = gamma dq, the
// energy E = sum P*H0 + 1/2 dq^T Q, delta q_max = max |q - q_prev|
// (Section "Sparsity and numerical accuracy") and linear charge mixing.
#include "sscf_internal.h"

namespace sscf {

namespace {

__global__ void k_dq(int n, const double* __restrict__ q, const int* __restrict__ species, double q0O, double q0H,
                     double* __restrict__ dq) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) dq[a] = q[a] - (species[a] == 0 ? q0O : q0H);
}

// One CTA per cluster: its energy (band + Coulomb) and max |q - q_prev|,
// fixed-order reductions.
__global__ void k_cluster_reduce(const int* __restrict__ cl_mol0, const int* __restrict__ cl_nmol,
                                 const double* __restrict__ e_mol, const double* __restrict__ q,
                                 const double* __restrict__ q_prev, const double* __restrict__ dq,
                                 const double* __restrict__ Q, double* __restrict__ cl_E, double* __restrict__ cl_dq) {
    __shared__ double s_e[256], s_m[256];
    const int cl = blockIdx.x;
    const int m0 = cl_mol0[cl], nm = cl_nmol[cl];
    double e = 0.0, mx = 0.0;
    for (int m = threadIdx.x; m < nm; m += blockDim.x) e += e_mol[m0 + m];
    for (int a = threadIdx.x; a < 3 * nm; a += blockDim.x) {
        const int at = 3 * m0 + a;
        e += 0.5 * dq[at] * Q[at];
        mx = fmax(mx, fabs(q[at] - q_prev[at]));
    }
    s_e[threadIdx.x] = e;
    s_m[threadIdx.x] = mx;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            s_e[threadIdx.x] += s_e[threadIdx.x + off];
            s_m[threadIdx.x] = fmax(s_m[threadIdx.x], s_m[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cl_E[cl] = s_e[0];
        cl_dq[cl] = s_m[0];
    }
}

// One CTA: fixed-order reductions (deterministic) and the mixing update.
__global__ void k_finish(int n_atoms, int n_mol, int mix, double beta, const double* __restrict__ e_mol,
                         double* __restrict__ q, double* __restrict__ q_prev, const double* __restrict__ dq,
                         const double* __restrict__ Q, double* __restrict__ dq_in, double* __restrict__ Q_in,
                         DeviceScalars* sc) {
    __shared__ double s_band[1024], s_coul[1024], s_max[1024];
    double band = 0.0, coul = 0.0, mx = 0.0;
    for (int m = threadIdx.x; m < n_mol; m += blockDim.x) band += e_mol[m];
    for (int a = threadIdx.x; a < n_atoms; a += blockDim.x) {
        coul += dq[a] * Q[a];
        mx = fmax(mx, fabs(q[a] - q_prev[a]));
    }
    s_band[threadIdx.x] = band;
    s_coul[threadIdx.x] = coul;
    s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            s_band[threadIdx.x] += s_band[threadIdx.x + off];
            s_coul[threadIdx.x] += s_coul[threadIdx.x + off];
            s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc->e_band = s_band[0];
        sc->e_coul = 0.5 * s_coul[0];
        sc->energy = s_band[0] + 0.5 * s_coul[0];
        sc->dq_max = s_max[0];
        if (!isfinite(sc->energy)) atomicOr(&sc->err, kErrNonFinite);
    }
    // after a capacity error the step's MOs are the previous ones: keep the charges
    if (sc->err & (kErrCapacity | kErrSortSize)) return;
    for (int a = threadIdx.x; a < n_atoms; a += blockDim.x) {
        q_prev[a] = q[a];
        if (mix) {
            dq_in[a] = dq_in[a] + beta * (dq[a] - dq_in[a]);
            Q_in[a] = Q_in[a] + beta * (Q[a] - Q_in[a]);
        } else {
            dq_in[a] = dq[a];
            Q_in[a] = Q[a];
        }
    }
}

// stored tiles of C and occupied tiles among them (one thread per row block)
__global__ void k_count_tiles(int n_mol, int cap, int n_occ_tiles, const int* __restrict__ c_nt,
                              const int* __restrict__ c_tile, unsigned long long* __restrict__ out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long all = 0, occ = 0;
    if (r < n_mol) {
        const int n = c_nt[r];
        all = n;
        for (int s = 0; s < n; ++s)
            if (c_tile[(size_t)r * cap + s] < n_occ_tiles) ++occ;
    }
    for (int off = 16; off > 0; off >>= 1) {
        all += __shfl_xor_sync(0xffffffffu, all, off);
        occ += __shfl_xor_sync(0xffffffffu, occ, off);
    }
    if ((threadIdx.x & 31) == 0 && all) {
        atomicAdd(&out[0], all);
        atomicAdd(&out[1], occ);
    }
}

}  // namespace

cudaError_t launch_count_tiles(Ctx* c, unsigned long long* out) {
    c->n_launch += 1;
    k_count_tiles<<<(c->n_mol + 255) / 256, 256, 0, c->stream>>>(c->n_mol, c->cap, c->n_occ_tiles, c->d_c_nt[c->cur],
                                                                 c->d_c_tile[c->cur], out);
    return cudaGetLastError();
}

cudaError_t launch_charges_finish(Ctx* c, bool mix) {
    c->n_launch += 2;
    k_dq<<<(c->n_atoms + 255) / 256, 256, 0, c->stream>>>(c->n_atoms, c->d_q, c->d_species, c->prm.q0[0],
                                                         c->prm.q0[1], c->d_dq);
    cudaError_t e = launch_gamma(c, c->d_dq, c->d_Q);
    if (e != cudaSuccess) return e;
    k_cluster_reduce<<<c->n_clusters, 256, 0, c->stream>>>(c->d_cl_mol0, c->d_cl_nmol, c->d_e_mol, c->d_q, c->d_q_prev,
                                                          c->d_dq, c->d_Q, c->d_cl_E, c->d_cl_dq);
    c->n_launch += 1;
    k_finish<<<1, 1024, 0, c->stream>>>(c->n_atoms, c->n_mol, mix ? 1 : 0, c->prm.mix_beta, c->d_e_mol, c->d_q,
                                        c->d_q_prev, c->d_dq, c->d_Q, c->d_dq_in, c->d_Q_in, c->d_sc);
    return cudaGetLastError();
}

}  // namespace sscf
