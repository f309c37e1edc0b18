"""Pins of oracle B (the paper's sparse SCF steps) against independent facts.

* the Jacobi 2x2 closed form annihilates F_ij (Section "Partial
  diagonalization"; the second rotation line read as -s C_ki + c C_kj);
* colourings are proper (no group twice in one colour) and complete;
* schedules never put one MO twice in a level;
* the neighbour-restricted transform equals the brute-force dense product on
  the kept blocks, and the group map equals a brute-force distance scan;
* the guess is local, orthonormal per molecule, and exact for one molecule;
* orthonormalisation reaches eps/100 and, for occupied-only passes, keeps the
  occupied projector;
* rotations applied row by row equal rotations applied column by column
  (the property the row-local GPU kernel relies on);
* the whole loop reproduces the dense eigensolve to far below the SCF
  convergence error, the paper's accuracy claim (Table "num_accuracy").
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import dense, model, sparse
from synth import default_params, lattice_water

P = default_params()
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_rotation_annihilates_pair():
    rng = np.random.default_rng(1)
    for _ in range(200):
        Fii, Fjj = rng.uniform(-1, 0.3, 2)
        Fij = rng.uniform(-0.1, 0.1) * 10 ** rng.uniform(-6, 0)
        F = np.array([[Fii, Fij], [Fij, Fjj]])
        c, s = sparse.rotation_angle(Fii, Fjj, Fij)
        R = np.array([[c, -s], [s, c]])           # columns: new c_i, new c_j
        Fp = R.T @ F @ R
        assert abs(Fp[0, 1]) <= 1e-14 * max(1.0, abs(Fii), abs(Fjj))
        assert c * c + s * s == pytest.approx(1.0, abs=1e-15)
        assert abs(s) <= abs(c) + 1e-15              # small-angle root, |t| <= 1
    c, s = sparse.rotation_angle(-0.5, -0.5, 1e-3)   # p = 0: sgn(0) = +1, 45 degrees
    assert c == pytest.approx(np.sqrt(0.5)) and s == pytest.approx(np.sqrt(0.5))


def test_paper_rotation_line_as_printed_is_not_orthogonal():
    c, s = sparse.rotation_angle(-0.4, -0.1, 0.02)
    printed = np.array([[c, s], [s, -s]])  # C'_kj = -s C_kj + c C_ki (as printed)
    assert not np.allclose(printed.T @ printed, np.eye(2))


@pytest.fixture(scope="module")
def sys32():
    s = lattice_water(32, seed=0)
    return s, sparse.SparseSCF(s, P)


def test_group_map_brute_force(sys32):
    s, sc = sys32
    G = s.n_groups
    atoms_of = [np.nonzero(s.group_of_mol[s.mol_of_atom] == g)[0] for g in range(G)]
    for A in range(G):
        for B in range(G):
            d = np.sqrt(((s.xyz[atoms_of[A], None, :] - s.xyz[None, atoms_of[B], :]) ** 2).sum(-1))
            assert sc.st.group_nb[A, B] == (A == B or d.min() < P["group_cut"])


def test_colouring_proper_and_complete():
    rng = np.random.default_rng(3)
    for G in (5, 17, 40):
        nb = rng.random((G, G)) < 0.3
        nb = nb | nb.T
        np.fill_diagonal(nb, True)
        col, n_col = sparse.colour_group_graph(nb)
        seen = {}
        for (A, B), c in col.items():
            if A == B:
                assert c == 0
                continue
            assert nb[A, B] and c >= 1
            for g in (A, B):
                assert (g, c) not in seen, "group used twice in one colour"
                seen[(g, c)] = True
        edges = {(A, B) for A in range(G) for B in range(A + 1, G) if nb[A, B]}
        assert edges == {k for k in col if k[0] != k[1]}
        degree = nb.sum(1) - 1
        assert n_col - 1 <= 2 * degree.max() - 1


def test_rotation_schedule_levels_disjoint(sys32):
    s, sc = sys32
    st = sc.st
    rng = np.random.default_rng(0)
    occ, vir = np.arange(st.n_occ), np.arange(st.n_occ, st.n_mo)
    mask = st.group_nb[st.mo_group[occ][:, None], st.mo_group[vir][None, :]]
    sel = mask & (rng.random(mask.shape) < 0.5)
    order = sparse.rotation_schedule(st, sel)
    assert len(order) == sel.sum()
    level = None
    used = set()
    n_occ_g = np.array([o.size for o in st.occ_of_group])
    n_virt_g = np.array([v.size for v in st.virt_of_group])
    for i, j in order:
        A, B = st.mo_group[i], st.mo_group[j]
        key = (st.colour[A, B], (st.mo_local[i] + st.mo_local[j]) % max(n_occ_g[A], n_virt_g[B]))
        if key != level:
            level, used = key, set()
        assert i not in used and j not in used
        used.update((i, j))


def test_guess_local_and_orthonormal(sys32):
    s, sc = sys32
    C = sparse.initial_guess(s, sc.st, sc.H0, sc.S)
    for m in range(s.n_mol):
        mos = np.nonzero(np.abs(C[6 * m:6 * m + 6]).sum(0))[0]
        assert mos.size == 6
        assert np.count_nonzero(C[:, mos]) == np.count_nonzero(C[6 * m:6 * m + 6, mos])
        sig = C[:, mos].T @ sc.S @ C[:, mos]
        assert np.allclose(sig, np.eye(6), atol=1e-12)
    one = lattice_water(1)
    sc1 = sparse.SparseSCF(one, P)
    C1 = sparse.initial_guess(one, sc1.st, sc1.H0, sc1.S)
    w = scipy.linalg.eigvalsh(sc1.H0, sc1.S)
    assert np.allclose(np.diag(C1.T @ sc1.H0 @ C1), w, atol=1e-12)


def test_orthonormalise_reaches_tolerance_and_keeps_occ_projector(sys32):
    s, sc = sys32
    eps = 1e-6
    C = sparse.initial_guess(s, sc.st, sc.H0, sc.S)
    passes, eta = sparse.orthonormalise(C, sc.S, sc.st, "all", eps)
    sig = C.T @ sc.S @ C
    assert eta < eps / 100
    assert np.abs(sig - np.eye(sig.shape[0])).max() < 1e-6
    # occupied-only passes keep span(C_occ) (up to the 1e-3 eps truncation)
    rng = np.random.default_rng(2)
    no = sc.st.n_occ
    Co = C[:, :no] + 1e-3 * rng.standard_normal((C.shape[0], no)) * (C[:, :no] != 0)
    C2 = C.copy()
    C2[:, :no] = Co

    def projector(X):
        return X @ np.linalg.solve(X.T @ sc.S @ X, X.T)
    P0 = projector(Co)
    sparse.orthonormalise(C2, sc.S, sc.st, "occ", eps)
    assert np.abs(projector(C2[:, :no]) - P0).max() < 1e-6
    assert np.abs(C2[:, :no].T @ sc.S @ C2[:, :no] - np.eye(no)).max() < 1e-6


def test_transform_matches_dense_product(sys32):
    s, sc = sys32
    st = sc.st
    rng = np.random.default_rng(4)
    C = rng.standard_normal((6 * s.n_mol, st.n_mo)) * (rng.random((6 * s.n_mol, st.n_mo)) < 0.4)
    H = sparse.fock(sc.H0, sc.S, rng.normal(0, 0.05, s.n_atoms), sc.atom_of_ao, 1e-6)
    F_ov, Fd, mask = sparse.transform_ov(C, H, st)
    for _ in range(300):
        i = rng.integers(st.n_occ)
        j = rng.integers(st.n_occ, st.n_mo)
        ref = sum(C[m, i] * H[m, n] * C[n, j] for m in range(C.shape[0]) for n in range(C.shape[0])
                  if H[m, n] != 0.0)
        if st.group_nb[st.mo_group[i], st.mo_group[j]]:
            assert F_ov[i, j - st.n_occ] == pytest.approx(ref, rel=1e-10, abs=1e-13)
        else:
            assert F_ov[i, j - st.n_occ] == 0.0
    k = rng.integers(st.n_mo)
    assert Fd[k] == pytest.approx(C[:, k] @ H @ C[:, k], rel=1e-12)


def test_fock_threshold_keeps_diagonal():
    s = lattice_water(4)
    sc = sparse.SparseSCF(s, P)
    H = sparse.fock(sc.H0, sc.S, np.zeros(s.n_atoms), sc.atom_of_ao, 0.01)
    off = H - np.diag(np.diag(H))
    assert np.all((off == 0) | (np.abs(off) >= 0.01))
    assert np.array_equal(np.diag(H), np.diag(sc.H0))


def test_select_pairs_cap_and_ties():
    F = np.array([[0.5, -0.3, 0.2], [0.3, 1e-7, -0.2], [0.0, 0.05, 0.2]])
    mask = np.ones_like(F, dtype=bool)
    mask[0, 0] = False
    sel = sparse.select_pairs(F, mask, 1e-6, 3)
    # candidates >= 1e-6 in mask: 0.3, 0.2, 0.3, 0.2, 0.05, 0.2 -> 3rd largest is 0.2, ties kept
    assert sel.sum() == 5
    assert not sel[0, 0] and not sel[1, 1] and not sel[2, 0] and not sel[2, 1]
    assert sparse.select_pairs(F, mask, 1e-6, 100).sum() == 6


def test_row_local_application_equals_column_sequential(sys32):
    s, sc = sys32
    st = sc.st
    rng = np.random.default_rng(5)
    C = sparse.initial_guess(s, st, sc.H0, sc.S)
    sparse.orthonormalise(C, sc.S, st, "all", 1e-4)
    H = sparse.fock(sc.H0, sc.S, np.zeros(s.n_atoms), sc.atom_of_ao, 1e-6)
    F_ov, Fd, mask = sparse.transform_ov(C, H, st)
    sel = sparse.select_pairs(F_ov, mask, 1e-6, 10 * st.n_occ)
    Ccol = C.copy()
    sparse.rotate_sweep(Ccol, F_ov, Fd, st, sel, 1e-6)
    order = sparse.rotation_schedule(st, sel)
    angles = [sparse.rotation_angle(Fd[i], Fd[j], F_ov[i, j - st.n_occ]) for i, j in order]
    Crow = C.copy()
    for k in rng.permutation(C.shape[0])[:60]:
        row = Crow[k]
        for (i, j), (c, sn) in zip(order, angles):
            ci, cj = row[i], row[j]
            a, b = c * ci + sn * cj, -sn * ci + c * cj
            row[i] = a if abs(a) >= 1e-6 else 0.0
            row[j] = b if abs(b) >= 1e-6 else 0.0
        assert np.array_equal(row, Ccol[k])


def test_sweep_is_orthogonal_without_truncation(sys32):
    s, sc = sys32
    st = sc.st
    C = sparse.initial_guess(s, st, sc.H0, sc.S)
    sparse.orthonormalise(C, sc.S, st, "all", 1e-6)
    H = sparse.fock(sc.H0, sc.S, np.zeros(s.n_atoms), sc.atom_of_ao, 1e-6)
    F_ov, Fd, mask = sparse.transform_ov(C, H, st)
    sel = sparse.select_pairs(F_ov, mask, 1e-6, 10 * st.n_occ)
    C2 = C.copy()
    sparse.rotate_sweep(C2, F_ov, Fd, st, sel, 0.0)
    Rm = np.linalg.lstsq(C, C2, rcond=None)[0]
    assert np.abs(Rm.T @ Rm - np.eye(Rm.shape[0])).max() < 1e-10
    # the sweep lowers the band energy of the occupied space
    no = st.n_occ
    assert np.trace(C2[:, :no].T @ H @ C2[:, :no]) < np.trace(C[:, :no].T @ H @ C[:, :no])


@pytest.mark.slow
def test_sparse_scf_matches_dense_below_scf_error():
    """Paper's accuracy claim (Table "num_accuracy"): the cut-off error stays
    below the error left by the SCF convergence criterion."""
    with open(os.path.join(GOLDEN, "paper_accuracy_table.json")) as f:
        table = json.load(f)
    worst_rel_1e5 = max(r["rel_error"] for r in table["dq_1e-5"])
    s = lattice_water(32, seed=0)
    ref = dense.solve(s, P)
    loose = dense.solve(s, P, dq_tol=1e-5, e_tol=1e-8)   # SCF stopped at the same criterion
    scf_error = abs(loose.energy - ref.energy)
    r = sparse.SparseSCF(s, P).run(eps=1e-6, dq_tol=1e-5, e_tol=1e-8)
    assert r["converged"]
    err = abs(r["energy"] - ref.energy)
    assert err < 1e-6 * s.n_atoms                 # 1e-6 Ha per atom target
    assert err < max(scf_error, 1e-9 * s.n_atoms)
    assert err / abs(ref.energy) < 100 * worst_rel_1e5
    assert np.abs(r["q"] - ref.q).max() < 1e-4


@pytest.mark.slow
@pytest.mark.parametrize("n", [8, 32])
def test_sparse_scf_without_cutoff_equals_dense(n):
    """The limit eps -> 0 of Section "Sparsity and numerical accuracy": with
    nothing truncated and every coupling rotated, the sparse SCF reaches the
    dense generalised-eigensolve ground state. The eps / 100 orthonormalisation
    target is zero there, so it is floored at 1e-13 (FP64 resolution of the
    normalised overlaps)."""
    s = lattice_water(n, seed=0)
    ref = dense.solve(s, P, dq_tol=1e-11, e_tol=1e-13)
    assert ref.converged
    r = sparse.SparseSCF(s, P, ortho_tol_min=1e-13).run(eps=0.0, dq_tol=1e-10, e_tol=1e-12)
    assert r["converged"]
    assert abs(r["energy"] - ref.energy) / s.n_atoms < 1e-10
    assert np.abs(r["q"] - ref.q).max() < 1e-8


def _landing(n, iters=40, eps=1e-3):
    """Oracle B's state after `iters` loose-stage SCC iterations, against oracle A."""
    s = lattice_water(n, seed=0)
    sc = sparse.SparseSCF(s, P)
    st = sc.start(eps)
    E = [sc.step(st, eps).energy for _ in range(iters)]
    A = dense.solve(s, P)
    no = sc.st.n_occ
    H = model.scc_hamiltonian(sc.H0, sc.S, st.Q_in, sc.atom_of_ao)
    F = st.C.T @ H @ st.C
    d = np.diag(F)
    Pb = model.density(st.C[:, :no])
    D = (Pb - A.P) @ sc.S
    return dict(n_atoms=s.n_atoms, E=E, E_A=A.energy, gap_A=A.gap, fov=float(np.abs(F[:no, no:]).max()),
                non_aufbau=int((d[:no] > d[no:].min()).sum()),
                proj=float(np.sqrt(np.trace(D @ D)) / (2 * no)))


@pytest.mark.slow
def test_small_gap_drives_the_sweeps_into_a_non_aufbau_state():
    """Where this synthetic model's SCC gap closes (dense HOMO-LUMO gap below
    ~0.04 Ha from ~70 molecules on), the paper's occupied-virtual Jacobi
    sweeps do not reach the dense ground state. The small-angle root of
    Section "Partial diagonalization" (|t| <= 1) never exchanges an occupied
    and a virtual MO, so once SCC transients lift occupied MOs above virtual
    ones the sweeps keep those occupations: the SCC runs uphill into a
    non-Aufbau state and keeps oscillating there, with couplings far above
    the threshold. At 48 molecules (gap 0.045 Ha) the same loose stage lands
    on the dense state within its truncation error."""
    ok = _landing(48)
    assert ok["gap_A"] > 0.04
    assert abs(ok["E"][-1] - ok["E_A"]) / ok["n_atoms"] < 2e-4
    assert ok["non_aufbau"] == 0
    assert ok["fov"] < 2e-3
    bad = _landing(72)
    assert bad["gap_A"] < 0.035
    assert bad["E"][-1] - bad["E_A"] > 1.0                    # Ha above the ground state
    assert bad["E"][-1] > bad["E"][9]                           # the SCC ran uphill
    assert bad["non_aufbau"] > 0.5 * 4 * 72                     # most occupied MOs above the lowest virtual
    assert bad["fov"] > 10 * 1e-3                               # not stationary at the sweep threshold
    assert bad["proj"] > 5 * ok["proj"]                         # a different occupied space
