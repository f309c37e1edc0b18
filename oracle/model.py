"""Synthetic SCC-DFTB model (oracle side, FP64, plain numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Section "Specific implementation for DFTB":
* Eq. (H_dftb) / (H_dftb2): H_mn = H0_mn + 1/2 S_mn (Q_a + Q_b), Q = gamma dq;
* Eq. (pop): q_a = sum_{m in a} sum_n P_mn S_mn with P = 2 C_occ C_occ^T;
* H0 and S come from two-centre Slater-Koster tables; here the tables are the
  synthetic V(r) = V0 exp(-r / r_decay) with a hard cut-off (r <= r_cut).

The energy E = sum P*H0 + 1/2 dq^T gamma dq is the standard second-order
SCC-DFTB energy; its derivative with respect to P is exactly the Hamiltonian
of Eq. (H_dftb) (pinned by a finite-difference test).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

N_AO_OF_SPECIES = (4, 1)   # O: s, px, py, pz; H: s


def ao_layout(species: np.ndarray):
    """First AO of every atom and the owning atom of every AO."""
    n_of = np.array(N_AO_OF_SPECIES)[species]
    first = np.concatenate([[0], np.cumsum(n_of)[:-1]])
    atom_of_ao = np.repeat(np.arange(species.size), n_of)
    return first, atom_of_ao, int(n_of.sum())


def dist2(xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """Squared distance evaluated as (dx*dx + dy*dy) + dz*dz, no fused ops."""
    d = xb - xa
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def atom_pairs_within(xyz: np.ndarray, r_cut: float):
    """All ordered atom pairs (a, b), a != b, with r_ab <= r_cut (brute force)."""
    n = xyz.shape[0]
    rows, cols = [], []
    rc2 = r_cut * r_cut
    chunk = 2048
    for s in range(0, n, chunk):
        d2 = dist2(xyz[s:s + chunk, None, :], xyz[None, :, :])
        a, b = np.nonzero(d2 <= rc2)
        a = a + s
        keep = a != b
        rows.append(a[keep])
        cols.append(b[keep])
    return np.concatenate(rows), np.concatenate(cols)


def sk_block(sa: int, sb: int, R: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Two-centre Slater-Koster block between atom a (bra) and atom b (ket).

    R = x_b - x_a; V = (ss-sigma, sp-sigma, pp-sigma, pp-pi) at r = |R|.
    Standard Slater-Koster direction-cosine rules (l, m, n) = R / r:
    <s|s> = Vss, <s|p_k> = e_k Vsp, <p_k|s> = -e_k Vsp,
    <p_k|p_k'> = e_k e_k' (Vpps - Vppp) + delta_kk' Vppp.
    """
    r = np.sqrt(dist2(np.zeros(3), R))
    e = R / r
    Vss, Vsp, Vpps, Vppp = V
    na, nb = N_AO_OF_SPECIES[sa], N_AO_OF_SPECIES[sb]
    B = np.zeros((na, nb))
    B[0, 0] = Vss
    if nb == 4:
        B[0, 1:4] = e * Vsp
    if na == 4:
        B[1:4, 0] = -e * Vsp
    if na == 4 and nb == 4:
        B[1:4, 1:4] = np.outer(e, e) * (Vpps - Vppp) + np.eye(3) * Vppp
    return B


def onsite_h0(species: int, p: dict) -> np.ndarray:
    if species == 0:
        return np.array([p["onsite_O_s"], p["onsite_O_p"], p["onsite_O_p"], p["onsite_O_p"]])
    return np.array([p["onsite_H_s"]])


def build_h0_s(sys, p: dict, dense: bool = True):
    """H0 and S on the atom-neighbour pattern (dense arrays or CSR).

    Every atom pair with r <= r_cut gets the Slater-Koster block of
    ``sk_block``; this routine evaluates the same rules for all pairs at once
    (element by element over the 4x4 orbital grid) and is pinned against
    ``sk_block`` in the tests.
    """
    first, atom_of_ao, n_ao = ao_layout(sys.species)
    rows = [first[a] + k for a in range(sys.n_atoms) for k in range(N_AO_OF_SPECIES[sys.species[a]])]
    rows = np.asarray(rows, dtype=np.int64)
    diag_h = np.concatenate([onsite_h0(int(s), p) for s in sys.species])
    R_list, C_list, H_list, S_list = [rows], [rows], [diag_h], [np.ones(rows.size)]
    pa, pb = atom_pairs_within(sys.xyz, p["r_cut"])
    R = sys.xyz[pb] - sys.xyz[pa]
    r = np.sqrt(dist2(np.zeros(3), R))
    e = R / r[:, None]
    decay = np.exp(-r / p["r_decay"])
    sa, sb = sys.species[pa], sys.species[pb]
    na = np.array(N_AO_OF_SPECIES)[sa]
    nb = np.array(N_AO_OF_SPECIES)[sb]
    for tab, out in ((np.asarray(p["V0"], float), H_list), (np.asarray(p["S0"], float), S_list)):
        Vss, Vsp, Vpps, Vppp = (tab[k] * decay for k in range(4))
        for i in range(4):
            for j in range(4):
                m = (i < na) & (j < nb)
                if i == 0 and j == 0:
                    v = Vss
                elif i == 0:
                    v = e[:, j - 1] * Vsp
                elif j == 0:
                    v = -e[:, i - 1] * Vsp
                else:
                    v = e[:, i - 1] * e[:, j - 1] * (Vpps - Vppp) + (Vppp if i == j else 0.0)
                out.append(v[m])
                if out is H_list:
                    R_list.append(first[pa[m]] + i)
                    C_list.append(first[pb[m]] + j)
    rr = np.concatenate(R_list)
    cc = np.concatenate(C_list)
    H0 = sp.csr_matrix((np.concatenate(H_list), (rr, cc)), shape=(n_ao, n_ao))
    S = sp.csr_matrix((np.concatenate(S_list), (rr, cc)), shape=(n_ao, n_ao))
    if dense:
        return H0.toarray(), S.toarray()
    return H0, S


def gamma_matrix(sys, p: dict) -> np.ndarray:
    """gamma_ab = 1 / sqrt(r^2 + a^2), a = (1/U_a + 1/U_b) / 2 (gamma_aa = U_a)."""
    U = np.where(sys.species == 0, p["U_O"], p["U_H"])
    inv = 1.0 / U
    a = 0.5 * (inv[:, None] + inv[None, :])
    d2 = dist2(sys.xyz[:, None, :], sys.xyz[None, :, :])
    return 1.0 / np.sqrt(d2 + a * a)


def gamma_times(sys, p: dict, dq: np.ndarray, chunk: int = 1024) -> np.ndarray:
    """Q = gamma dq without storing gamma (for clusters too large for it)."""
    U = np.where(sys.species == 0, p["U_O"], p["U_H"])
    inv = 1.0 / U
    out = np.empty(sys.n_atoms)
    for s in range(0, sys.n_atoms, chunk):
        a = 0.5 * (inv[s:s + chunk, None] + inv[None, :])
        d2 = dist2(sys.xyz[s:s + chunk, None, :], sys.xyz[None, :, :])
        out[s:s + chunk] = (1.0 / np.sqrt(d2 + a * a)) @ dq
    return out


def reference_population(sys, p: dict) -> np.ndarray:
    return np.where(sys.species == 0, p["q0_O"], p["q0_H"]).astype(np.float64)


def scc_hamiltonian(H0, S, Q: np.ndarray, atom_of_ao: np.ndarray):
    """Eq. (H_dftb2): H_mn = H0_mn + 1/2 S_mn (Q_a + Q_b)."""
    Qao = Q[atom_of_ao]
    if sp.issparse(S):
        S = S.tocoo()
        vals = S.data * 0.5 * (Qao[S.row] + Qao[S.col])
        return (H0 + sp.csr_matrix((vals, (S.row, S.col)), shape=S.shape)).tocsr()
    return H0 + 0.5 * S * (Qao[:, None] + Qao[None, :])


def density(C_occ: np.ndarray) -> np.ndarray:
    """P = sum_i n_i c_i c_i^T with n_i = 2 for every occupied MO (Eq. pop)."""
    return 2.0 * C_occ @ C_occ.T


def mulliken(P, S, atom_of_ao: np.ndarray, n_atoms: int) -> np.ndarray:
    """Eq. (pop): q_a = sum_{m in a} sum_n P_mn S_mn."""
    if sp.issparse(S):
        S = S.tocoo()
        contrib = np.asarray(P[S.row, S.col]).ravel() * S.data
        per_ao = np.bincount(S.row, weights=contrib, minlength=S.shape[0])
    else:
        per_ao = (P * S).sum(axis=1)
    return np.bincount(atom_of_ao, weights=per_ao, minlength=n_atoms)


def energy(P, H0, dq: np.ndarray, Q: np.ndarray) -> float:
    """Second-order SCC energy E = sum_mn P_mn H0_mn + 1/2 dq^T Q, Q = gamma dq."""
    if sp.issparse(H0):
        H0 = H0.tocoo()
        band = float(np.dot(np.asarray(P[H0.row, H0.col]).ravel(), H0.data))
    else:
        band = float((P * H0).sum())
    return band + 0.5 * float(dq @ Q)
