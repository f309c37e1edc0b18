"""Oracle B: the paper's sparse SCF algorithm, step by step, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

MO coefficients live in a dense (N_AO x N_MO) float64 array whose zeros are
the sparsity pattern; every truncation writes exact zeros. The steps follow
the paper's Sections in order:

I    neighbour lists of atoms and of MO groups (Section "Defining
     neighbouring lists"), plus the colouring of the MO-group graph that
     orders block-parallel work (Figure "jacobi");
II   initial guess: one non-SCC generalised eigensolve per molecule
     (Section "Initial guess");
III  orthonormalisation by normalisation plus pairwise first-order
     combinations (Section "Orthonormalization", steps a-e);
IV   DFTB Hamiltonian Eq. (H_dftb2), Mulliken charges Eq. (pop);
V    partial diagonalisation: Jacobi rotations on occupied-virtual pairs
     (Section "Partial diagonalization", steps 1-4), angles from the
     C^T H C values at the start of the sweep.

Readings where the paper is silent or garbled (each also listed in the design
notes): the second rotation line is C'_kj = -s C_ki + c C_kj; sgn(0) = +1;
all pairs of one sweep use the F values of the sweep start; at most
10 N_occ rotations per sweep, the largest |F_ij| first (ties at the cut kept);
pairs are applied colour by colour, block colour first, then the in-block
colour (i_loc + j_loc) mod n; orthonormalisation combinations use the
normalised overlap of the pass start for both MOs simultaneously;
truncation (|C| < threshold -> 0) follows every 2x2 update.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from . import model


# --------------------------------------------------------------------------
# Step I: structure
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Structure:
    n_mol: int
    n_groups: int
    group_of_mol: np.ndarray
    mols_of_group: list            # sorted molecule ids per group
    occ_of_group: list             # global occupied MO ids per group
    virt_of_group: list            # global virtual MO ids per group
    mo_group: np.ndarray           # group of every MO
    mo_local: np.ndarray           # index inside the group's occ (or virt) list
    mo_is_occ: np.ndarray
    group_nb: np.ndarray           # (n_groups, n_groups) bool, True for neighbours and A == B
    edge_colour: dict              # (A, B), A <= B -> colour (0 for A == B)
    colour: np.ndarray             # (n_groups, n_groups) symmetric colour matrix, -1 off the graph
    n_colours: int
    n_occ: int
    n_mo: int


def group_neighbours(sys, group_cut: float) -> np.ndarray:
    """Two groups are neighbours if some atom pair between them is closer than group_cut."""
    g_of_atom = sys.group_of_mol[sys.mol_of_atom]
    G = sys.n_groups
    nb = np.zeros((G, G), dtype=bool)
    gc2 = group_cut * group_cut
    chunk = 1024
    for s in range(0, sys.n_atoms, chunk):
        d2 = model.dist2(sys.xyz[s:s + chunk, None, :], sys.xyz[None, :, :])
        a, b = np.nonzero(d2 < gc2)
        nb[g_of_atom[a + s], g_of_atom[b]] = True
    np.fill_diagonal(nb, True)
    return nb


def colour_group_graph(nb: np.ndarray):
    """Greedy first-fit edge colouring of the MO-group graph.

    Edges {A, B}, A < B, are visited in lexicographic order and take the
    smallest colour >= 1 used by no edge already coloured at A or at B.
    Every self pair (A, A) has colour 0. Blocks of one colour share no group,
    which is the property the block-parallel schedule of Figure "jacobi" needs.
    """
    G = nb.shape[0]
    used = [set() for _ in range(G)]
    colour = {}
    n_col = 1
    for A in range(G):
        colour[(A, A)] = 0
        for B in range(A + 1, G):
            if not nb[A, B]:
                continue
            c = 1
            while c in used[A] or c in used[B]:
                c += 1
            colour[(A, B)] = c
            used[A].add(c)
            used[B].add(c)
            n_col = max(n_col, c + 1)
    return colour, n_col


def build_structure(sys, p: dict) -> Structure:
    G = sys.n_groups
    mols_of_group = [np.sort(np.nonzero(sys.group_of_mol == g)[0]) for g in range(G)]
    n_mol = sys.n_mol
    n_occ = 4 * n_mol
    occ_of_group, virt_of_group = [], []
    o, v = 0, n_occ
    for g in range(G):
        k = mols_of_group[g].size
        occ_of_group.append(np.arange(o, o + 4 * k))
        virt_of_group.append(np.arange(v, v + 2 * k))
        o += 4 * k
        v += 2 * k
    n_mo = 6 * n_mol
    mo_group = np.empty(n_mo, dtype=np.int64)
    mo_local = np.empty(n_mo, dtype=np.int64)
    mo_is_occ = np.zeros(n_mo, dtype=bool)
    for g in range(G):
        mo_group[occ_of_group[g]] = g
        mo_local[occ_of_group[g]] = np.arange(occ_of_group[g].size)
        mo_is_occ[occ_of_group[g]] = True
        mo_group[virt_of_group[g]] = g
        mo_local[virt_of_group[g]] = np.arange(virt_of_group[g].size)
    nb = group_neighbours(sys, p["group_cut"])
    colour, n_col = colour_group_graph(nb)
    cmat = -np.ones((G, G), dtype=np.int64)
    for (A, B), c in colour.items():
        cmat[A, B] = cmat[B, A] = c
    return Structure(n_mol=n_mol, n_groups=G, group_of_mol=sys.group_of_mol,
                     mols_of_group=mols_of_group, occ_of_group=occ_of_group,
                     virt_of_group=virt_of_group, mo_group=mo_group, mo_local=mo_local,
                     mo_is_occ=mo_is_occ, group_nb=nb, edge_colour=colour,
                     colour=cmat, n_colours=n_col, n_occ=n_occ, n_mo=n_mo)


# --------------------------------------------------------------------------
# Step II: initial guess
# --------------------------------------------------------------------------

def fix_sign(v: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude coefficient positive (first index within 1e-9 of the max)."""
    a = np.abs(v)
    k = int(np.nonzero(a >= a.max() * (1.0 - 1e-9))[0][0])
    return v if v[k] > 0 else -v


def initial_guess(sys, st: Structure, H0: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Per-molecule non-SCC solve; occupied MOs group-major, then virtual MOs.

    Within a molecule the MOs follow ascending eigenvalue; the four lowest are
    occupied (8 valence electrons per water molecule).
    """
    n_ao = 6 * sys.n_mol
    C = np.zeros((n_ao, st.n_mo))
    for g in range(st.n_groups):
        for k, m in enumerate(st.mols_of_group[g]):
            sl = slice(6 * m, 6 * m + 6)
            w, V = scipy.linalg.eigh(H0[sl, sl], S[sl, sl])
            for n in range(6):
                vec = fix_sign(V[:, n])
                if n < 4:
                    C[sl, st.occ_of_group[g][4 * k + n]] = vec
                else:
                    C[sl, st.virt_of_group[g][2 * k + n - 4]] = vec
    return C


# --------------------------------------------------------------------------
# Step III: orthonormalisation
# --------------------------------------------------------------------------

def pass_mos(st: Structure, which: str, g: int) -> np.ndarray:
    """MOs of group g taking part in an orthonormalisation pass (occupied first)."""
    if which == "occ":
        return st.occ_of_group[g]
    return np.concatenate([st.occ_of_group[g], st.virt_of_group[g]])


def pass_local(st: Structure, which: str, mos: np.ndarray) -> np.ndarray:
    """Index of each MO inside its group's list for the pass (occupied first)."""
    loc = st.mo_local[mos].copy()
    if which != "occ":
        n_occ_g = np.array([o.size for o in st.occ_of_group])
        virt = ~st.mo_is_occ[mos]
        loc[virt] += n_occ_g[st.mo_group[mos][virt]]
    return loc


def pass_group_size(st: Structure, which: str) -> np.ndarray:
    return np.array([pass_mos(st, which, g).size for g in range(st.n_groups)])


def ortho_schedule(st: Structure, which: str, mos: np.ndarray, sel: np.ndarray):
    """Selected pairs (positions into ``mos``) in schedule order.

    ``sel`` is a boolean matrix over pairs of ``mos``; only pairs whose first
    MO sits in the lower group (or, inside one group, has the lower local
    index) are scheduled. Order: colour of the block (A, B), then in-block
    colour (i_loc + j_loc) mod max(n_A, n_B), then i, then j.
    """
    g = st.mo_group[mos]
    loc = pass_local(st, which, mos)
    a, b = np.nonzero(sel)
    ga, gb = g[a], g[b]
    first = (ga < gb) | ((ga == gb) & (loc[a] < loc[b]))
    a, b, ga, gb = a[first], b[first], ga[first], gb[first]
    size = pass_group_size(st, which)
    n = np.maximum(size[ga], size[gb])
    col = st.colour[ga, gb]
    sub = (loc[a] + loc[b]) % n
    order = np.lexsort((mos[b], mos[a], sub, col))
    return a[order], b[order]


def overlap_mask(st: Structure, mos: np.ndarray) -> np.ndarray:
    """Pairs of MOs in neighbouring (or equal) groups: only those blocks of C^T X C are kept."""
    g = st.mo_group[mos]
    return st.group_nb[g[:, None], g[None, :]]


def truncate(v: np.ndarray, thr: float) -> np.ndarray:
    v[np.abs(v) < thr] = 0.0
    return v


def ortho_pass(C: np.ndarray, S: np.ndarray, st: Structure, which: str,
               tol: float, trunc: float, sigma: np.ndarray | None = None):
    """One pass of steps b-d; returns (eta, number of combinations).

    A pass that finds eta below the target has found the MOs orthonormal: it
    ends the orthonormalisation (step e) without normalising again.

    ``sigma`` (optional) supplies the overlaps of step b instead of computing
    them, so that steps c-d can be checked alone on given overlaps.
    """
    mos = np.arange(st.n_occ) if which == "occ" else np.arange(st.n_mo)
    Cm = C[:, mos]
    if sigma is None:
        sigma = Cm.T @ (S @ Cm)                  # step b: C^T S C
    sigma = np.where(overlap_mask(st, mos), sigma, 0.0)
    d = np.sqrt(np.diag(sigma))
    sig_n = sigma / np.outer(d, d)
    off = np.abs(sig_n - np.diag(np.diag(sig_n)))
    eta = float(off.max()) if off.size else 0.0
    if eta < tol:
        return eta, 0                            # converged: the pass changes nothing
    C[:, mos] = Cm / d[None, :]                  # step c: normalise
    sel = overlap_mask(st, mos) & (np.abs(sig_n) >= 1e-3 * eta)
    np.fill_diagonal(sel, False)
    pa, pb = ortho_schedule(st, which, mos, sel)
    for a, b in zip(pa.tolist(), pb.tolist()):   # step d: first-order combinations
        s = sig_n[a, b]
        i, j = mos[a], mos[b]
        ci, cj = C[:, i].copy(), C[:, j].copy()
        C[:, i] = truncate(ci - 0.5 * s * cj, trunc)
        C[:, j] = truncate(cj - 0.5 * s * ci, trunc)
    return eta, int(pa.size)


def orthonormalise(C, S, st, which: str, eps: float, max_pass: int = 200, tol_min: float = 0.0):
    """Repeat passes until the largest off-diagonal overlap is below eps / 100.

    Combinations truncate at 1e-3 eps (Section "Sparsity and numerical accuracy").
    ``tol_min`` is a floor under the eps / 100 target; it matters only where
    eps / 100 lies below what the arithmetic can resolve (eps -> 0, where the
    target would be zero).
    """
    tol = max(eps / 100.0, tol_min)
    trunc = 1e-3 * eps
    for k in range(1, max_pass + 1):
        eta, n = ortho_pass(C, S, st, which, tol, trunc)
        if eta < tol:
            return k, eta
    return max_pass, eta


# --------------------------------------------------------------------------
# Step IV: Hamiltonian, charges, energy
# --------------------------------------------------------------------------

def fock(H0, S, Q, atom_of_ao, eps: float) -> np.ndarray:
    """Eq. (H_dftb2) with off-diagonal elements |H_mn| < eps set to zero."""
    H = model.scc_hamiltonian(H0, S, Q, atom_of_ao)
    small = np.abs(H) < eps
    np.fill_diagonal(small, False)
    H = H.copy()
    H[small] = 0.0
    return H


# --------------------------------------------------------------------------
# Step V: partial diagonalisation
# --------------------------------------------------------------------------

def transform_ov(C, H, st: Structure):
    """F = C^T H C on occupied-virtual blocks of neighbouring groups, and diag(F)."""
    HC = H @ C
    F = C.T @ HC
    occ = np.arange(st.n_occ)
    vir = np.arange(st.n_occ, st.n_mo)
    go, gv = st.mo_group[occ], st.mo_group[vir]
    mask = st.group_nb[go[:, None], gv[None, :]]
    F_ov = np.where(mask, F[np.ix_(occ, vir)], 0.0)
    return F_ov, np.diag(F).copy(), mask


def select_pairs(F_ov, mask, tau: float, k_max: int):
    """Pairs with |F_ij| >= tau; at most k_max of the largest (ties at the cut kept)."""
    a = np.abs(F_ov)
    cand = mask & (a >= tau)
    vals = a[cand]
    if vals.size > k_max:
        v_k = np.sort(vals)[::-1][k_max - 1]
        cand = cand & (a >= v_k)
    return cand


def rotation_angle(Fii: float, Fjj: float, Fij: float):
    """Jacobi angle of Section "Partial diagonalization": p, t, c, s (sgn(0) = +1)."""
    p = (Fii - Fjj) / (2.0 * Fij)
    sg = 1.0 if p >= 0.0 else -1.0
    t = 1.0 / (p + sg * np.sqrt(1.0 + p * p))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, t * c


def rotation_schedule(st: Structure, sel: np.ndarray):
    """Selected (i, j) pairs in schedule order.

    Block (A occ, B virt) has the colour of edge {A, B} (0 for A == B); inside
    a block, pairs go by (i_loc + j_loc) mod max(n_occ(A), n_virt(B)).
    """
    oi, vj = np.nonzero(sel)
    i, j = oi, st.n_occ + vj
    A, B = st.mo_group[i], st.mo_group[j]
    n_occ_g = np.array([o.size for o in st.occ_of_group])
    n_virt_g = np.array([v.size for v in st.virt_of_group])
    col = st.colour[A, B]
    sub = (st.mo_local[i] + st.mo_local[j]) % np.maximum(n_occ_g[A], n_virt_g[B])
    order = np.lexsort((j, i, sub, col))
    return list(zip(i[order].tolist(), j[order].tolist()))


def rotate_sweep(C, F_ov, Fd, st: Structure, sel, trunc: float):
    """Apply the selected rotations in schedule order, truncating after each."""
    order = rotation_schedule(st, sel)
    for i, j in order:
        c, s = rotation_angle(Fd[i], Fd[j], F_ov[i, j - st.n_occ])
        ci, cj = C[:, i].copy(), C[:, j].copy()
        C[:, i] = truncate(c * ci + s * cj, trunc)
        C[:, j] = truncate(-s * ci + c * cj, trunc)
    return len(order)


# --------------------------------------------------------------------------
# SCC driver
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SparseState:
    C: np.ndarray
    dq_in: np.ndarray
    Q_in: np.ndarray
    q_prev: np.ndarray
    E_prev: float


@dataclasses.dataclass
class StepInfo:
    energy: float
    dq_max: float
    n_rot: int
    max_fov: float
    eta: float
    nnz_per_mo: float
    dE: float


class SparseSCF:
    """Plain sparse SCF on one cluster (oracle B)."""

    def __init__(self, sys, p: dict, ortho_every: int = 1, ortho_tol_min: float = 0.0):
        self.sys, self.p = sys, p
        self.ortho_every = ortho_every
        self.ortho_tol_min = ortho_tol_min   # floor under every eps / 100 target (see orthonormalise)
        self.first, self.atom_of_ao, self.n_ao = model.ao_layout(sys.species)
        self.H0, self.S = model.build_h0_s(sys, p, dense=True)
        self.G = model.gamma_matrix(sys, p)
        self.q0 = model.reference_population(sys, p)
        self.st = build_structure(sys, p)

    def charges_energy(self, C):
        P = model.density(C[:, :self.st.n_occ])
        q = model.mulliken(P, self.S, self.atom_of_ao, self.sys.n_atoms)
        dq = q - self.q0
        Q = self.G @ dq
        return q, dq, Q, model.energy(P, self.H0, dq, Q)

    def start(self, eps: float) -> SparseState:
        C = initial_guess(self.sys, self.st, self.H0, self.S)
        orthonormalise(C, self.S, self.st, "all", eps, tol_min=self.ortho_tol_min)
        q, dq, Q, E = self.charges_energy(C)
        return SparseState(C=C, dq_in=dq, Q_in=Q, q_prev=q, E_prev=E)

    def step(self, s: SparseState, eps: float) -> StepInfo:
        st, p = self.st, self.p
        H = fock(self.H0, self.S, s.Q_in, self.atom_of_ao, eps)
        F_ov, Fd, mask = transform_ov(s.C, H, st)
        k_max = int(p["rot_cap_factor"] * st.n_occ)
        sel = select_pairs(F_ov, mask, eps, k_max)
        n_rot = rotate_sweep(s.C, F_ov, Fd, st, sel, eps)
        eta = 0.0
        if self.ortho_every:
            tol = max(eps / 100.0, self.ortho_tol_min)
            eta, _ = ortho_pass(s.C, self.S, st, "occ", tol, 1e-3 * eps)
        q, dq, Q, E = self.charges_energy(s.C)
        dq_max = float(np.max(np.abs(q - s.q_prev)))
        beta = p["mix_beta"]
        s.dq_in = s.dq_in + beta * (dq - s.dq_in)
        s.Q_in = s.Q_in + beta * (Q - s.Q_in)
        dE = E - s.E_prev
        s.q_prev, s.E_prev = q, E
        info = StepInfo(energy=E, dq_max=dq_max, n_rot=n_rot,
                        max_fov=float(np.abs(F_ov).max()), eta=eta,
                        nnz_per_mo=float(np.count_nonzero(s.C)) / st.n_mo, dE=dE)
        return info

    def run(self, eps: float | None = None, dq_tol: float | None = None,
            e_tol: float | None = None, loose=(1e-3, 1e-1), max_iter: int | None = None,
            log=None):
        """Loose SCF, then the user thresholds, then the final occupied orthonormalisation."""
        p = self.p
        eps = p["eps_mo"] if eps is None else eps
        dq_tol = p["dq_tol"] if dq_tol is None else dq_tol
        e_tol = p["e_tol"] if e_tol is None else e_tol
        max_iter = p["max_scc"] if max_iter is None else max_iter
        stages = []
        if loose is not None:
            stages.append((loose[0], loose[1], np.inf))
        stages.append((eps, dq_tol, e_tol))
        s = self.start(stages[0][0])
        n_iter = 0
        converged = False
        for k, (eps_k, dq_k, e_k) in enumerate(stages):
            converged = False
            if k > 0:
                # the user-threshold SCF starts again from step III with the
                # improved MOs: full orthonormalisation at the new threshold
                orthonormalise(s.C, self.S, self.st, "all", eps_k, tol_min=self.ortho_tol_min)
            for _ in range(max_iter):
                info = self.step(s, eps_k)
                n_iter += 1
                if log is not None:
                    log(n_iter, eps_k, info)
                if info.dq_max <= dq_k and abs(info.dE) <= e_k:
                    converged = True
                    break
        orthonormalise(s.C, self.S, self.st, "occ", eps, tol_min=self.ortho_tol_min)
        q, dq, Q, E = self.charges_energy(s.C)
        return dict(energy=E, q=q, dq=dq, C=s.C, iterations=n_iter, converged=converged)
