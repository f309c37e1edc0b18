"""Analytic energy gradients at SCC convergence (oracle side, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper computes energies only; gradients are the adjoint of its energy
(Eq. H_dftb, Eq. pop) at the converged, orthonormal occupied space
(C^T S C = I, F_ov = 0):

    dE = sum P * dH0 + sum (1/2 P * (Q_a + Q_b) - W) * dS + 1/2 dq^T dgamma dq,

with W = 1/2 P H P the energy-weighted density (H the SCC Hamiltonian), the
Mulliken term coming from the explicit S dependence of Eq. (pop). Forces take
the derivatives of the Slater-Koster blocks and of gamma with respect to the
atom positions; parameter gradients use that H0 is linear in the V0 and S in
the S0 prefactors.
"""
from __future__ import annotations

import numpy as np

from . import model


def sk_block_grad(sa: int, sb: int, R: np.ndarray, V0: np.ndarray, r_decay: float) -> np.ndarray:
    """d(block)/dR_k for V(r) = V0 exp(-r / r_decay); returns (3, na, nb).

    Differentiates the direction-cosine rules of ``model.sk_block``:
    dV/dr = -V / r_decay, dr/dR_k = e_k, de_i/dR_k = (delta_ik - e_i e_k) / r.
    """
    r = float(np.sqrt(model.dist2(np.zeros(3), R)))
    e = R / r
    V = V0 * np.exp(-r / r_decay)
    dV = -V / r_decay                                  # dV/dr
    na, nb = model.N_AO_OF_SPECIES[sa], model.N_AO_OF_SPECIES[sb]
    out = np.zeros((3, na, nb))
    de = (np.eye(3) - np.outer(e, e)) / r              # de[i, k] = d e_i / d R_k
    for k in range(3):
        dVk = dV * e[k]
        out[k, 0, 0] = dVk[0]
        if nb == 4:
            out[k, 0, 1:4] = de[:, k] * V[1] + e * dVk[1]
        if na == 4:
            out[k, 1:4, 0] = -(de[:, k] * V[1] + e * dVk[1])
        if na == 4 and nb == 4:
            dee = np.outer(de[:, k], e) + np.outer(e, de[:, k])
            out[k, 1:4, 1:4] = dee * (V[2] - V[3]) + np.outer(e, e) * (dVk[2] - dVk[3]) + np.eye(3) * dVk[3]
    return out


def energy_weighted_density(P: np.ndarray, H: np.ndarray) -> np.ndarray:
    """W = 1/2 P H P (equals sum_i n_i e_i c_i c_i^T for canonical MOs)."""
    return 0.5 * P @ H @ P


def gradients(sys, p: dict, P: np.ndarray, dq: np.ndarray):
    """dE/dxyz (n_atoms, 3) and dE/d(V0[0..3], S0[0..3]) at a converged density P."""
    first, atom_of_ao, n_ao = model.ao_layout(sys.species)
    H0, S = model.build_h0_s(sys, p, dense=True)
    G = model.gamma_matrix(sys, p)
    Q = G @ dq
    H = model.scc_hamiltonian(H0, S, Q, atom_of_ao)
    W = energy_weighted_density(P, H)
    Qao = Q[atom_of_ao]
    GS = 0.5 * P * (Qao[:, None] + Qao[None, :]) - W   # contraction weight of dS
    grad = np.zeros((sys.n_atoms, 3))
    V0 = np.asarray(p["V0"], dtype=float)
    S0 = np.asarray(p["S0"], dtype=float)
    pa, pb = model.atom_pairs_within(sys.xyz, p["r_cut"])
    for a, b in zip(pa.tolist(), pb.tolist()):
        R = sys.xyz[b] - sys.xyz[a]
        sa, sb = int(sys.species[a]), int(sys.species[b])
        dH = sk_block_grad(sa, sb, R, V0, p["r_decay"])
        dS = sk_block_grad(sa, sb, R, S0, p["r_decay"])
        na, nb = dH.shape[1:]
        blkP = P[first[a]:first[a] + na, first[b]:first[b] + nb]
        blkG = GS[first[a]:first[a] + na, first[b]:first[b] + nb]
        g = np.einsum("kij,ij->k", dH, blkP) + np.einsum("kij,ij->k", dS, blkG)
        grad[b] += g          # the block depends on R = x_b - x_a
        grad[a] -= g
    # 1/2 dq^T dgamma dq over ordered pairs, gamma = (r^2 + s^2)^(-1/2)
    D = sys.xyz[:, None, :] - sys.xyz[None, :, :]
    grad += -(dq[:, None, None] * dq[None, :, None] * (G ** 3)[:, :, None] * D).sum(axis=1)
    # parameters: H0 is linear in V0, S - I is linear in S0
    zero = dict(p, onsite_O_s=0.0, onsite_O_p=0.0, onsite_H_s=0.0)
    dpar = np.zeros(8)
    for k in range(4):
        unit = np.zeros(4)
        unit[k] = 1.0
        Hk, Sk = model.build_h0_s(sys, dict(zero, V0=tuple(unit), S0=tuple(unit)), dense=True)
        Sk = Sk - np.eye(n_ao)
        dpar[k] = float((P * Hk).sum())
        dpar[4 + k] = float((GS * Sk).sum())
    return grad, dpar
