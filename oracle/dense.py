"""Oracle A: the definition of the sparse SCF's result (FP64, dense).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The closed-shell SCC-DFTB ground state is the fixed point of
H[dq] C = S C e with the N_occ lowest MOs doubly occupied, H from
Eq. (H_dftb2) and dq from Eq. (pop). The paper validates its sparse method
against the LAPACK divide-and-conquer generalised eigensolver DSYGVD
(Table "num_accuracy"); this oracle runs the same solver (scipy's
``eigh(driver="gvd")``) inside a plain linearly mixed SCC loop.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from . import model


@dataclasses.dataclass
class DenseResult:
    energy: float
    q: np.ndarray
    dq: np.ndarray
    Q: np.ndarray
    C: np.ndarray
    eigenvalues: np.ndarray
    P: np.ndarray
    iterations: int
    converged: bool
    gap: float          # lowest virtual minus highest occupied eigenvalue (Ha)


def solve(sys, p: dict, dq_tol: float = 1e-10, e_tol: float = 1e-12,
          max_iter: int = 500, beta: float | None = None, H0S=None, gamma=None):
    """Dense SCC loop; returns energy, charges, MOs and the HOMO-LUMO gap."""
    first, atom_of_ao, n_ao = model.ao_layout(sys.species)
    H0, S = H0S if H0S is not None else model.build_h0_s(sys, p, dense=True)
    G = gamma if gamma is not None else model.gamma_matrix(sys, p)
    q0 = model.reference_population(sys, p)
    n_occ = 4 * sys.n_mol
    beta = p["mix_beta"] if beta is None else beta
    dq = np.zeros(sys.n_atoms)
    Q = G @ dq
    q_prev = None
    E_prev = None
    converged = False
    for it in range(1, max_iter + 1):
        H = model.scc_hamiltonian(H0, S, Q, atom_of_ao)
        w, C = scipy.linalg.eigh(H, S, driver="gvd")
        P = model.density(C[:, :n_occ])
        q = model.mulliken(P, S, atom_of_ao, sys.n_atoms)
        dq_out = q - q0
        Q_out = G @ dq_out
        E = model.energy(P, H0, dq_out, Q_out)
        if q_prev is not None:
            if np.max(np.abs(q - q_prev)) <= dq_tol and abs(E - E_prev) <= e_tol:
                converged = True
                break
        q_prev, E_prev = q, E
        dq = dq + beta * (dq_out - dq)
        Q = Q + beta * (Q_out - Q)
    return DenseResult(energy=E, q=q, dq=dq_out, Q=Q_out, C=C, eigenvalues=w, P=P,
                       iterations=it, converged=converged,
                       gap=float(w[n_occ] - w[n_occ - 1]))
