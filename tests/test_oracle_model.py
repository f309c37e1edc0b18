"""Pins of the oracle's model layer against closed forms and invariants.

Each test checks the oracle against something other than itself: a
Slater-Koster closed form for a chosen geometry, rotational invariance,
the limit of the SCC gamma, a finite-difference derivative of the energy
(which ties Eq. (H_dftb2) to the energy expression), and the charge sum.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import dense, model
from synth import default_params, lattice_water
from synth.water import WaterSystem


def _pair(species_a, species_b, R):
    xyz = np.array([[0.0, 0.0, 0.0], R], dtype=np.float64)
    species = np.array([species_a, species_b], dtype=np.int32)
    return WaterSystem(n_mol=1, species=species, xyz=xyz, mol_of_atom=np.zeros(2, np.int32),
                       site=np.zeros((1, 3), np.int32), group_of_mol=np.zeros(1, np.int32),
                       n_groups=1, lattice_edge=1)


P = default_params()


def V(k, r, table="V0"):
    return P[table][k] * np.exp(-r / P["r_decay"])


def test_sk_closed_form_along_x():
    r = 3.7
    sysm = _pair(0, 0, [r, 0.0, 0.0])
    H0, S = model.build_h0_s(sysm, P)
    B = H0[0:4, 4:8]
    assert B[0, 0] == pytest.approx(V(0, r))                 # s-s sigma
    assert B[0, 1] == pytest.approx(V(1, r))                 # s(a)-px(b): +l Vsp
    assert B[1, 0] == pytest.approx(-V(1, r))                # px(a)-s(b): -l Vsp
    assert B[1, 1] == pytest.approx(V(2, r))                 # px-px along the bond: pp sigma
    assert B[2, 2] == pytest.approx(V(3, r))                 # py-py: pp pi
    assert B[3, 3] == pytest.approx(V(3, r))
    assert B[1, 2] == 0.0 and B[0, 2] == 0.0
    Sb = S[0:4, 4:8]
    assert Sb[1, 1] == pytest.approx(V(2, r, "S0"))
    assert np.array_equal(S[0:4, 0:4], np.eye(4))
    assert np.allclose(np.diag(H0)[:4], [P["onsite_O_s"]] + [P["onsite_O_p"]] * 3)


def test_sk_closed_form_diagonal_direction():
    r = 4.0
    R = np.array([r / np.sqrt(2), r / np.sqrt(2), 0.0])
    H0, _ = model.build_h0_s(_pair(0, 0, R), P)
    B = H0[0:4, 4:8]
    assert B[1, 2] == pytest.approx(0.5 * (V(2, r) - V(3, r)))
    assert B[1, 1] == pytest.approx(0.5 * V(2, r) + 0.5 * V(3, r))
    assert B[0, 3] == pytest.approx(0.0, abs=1e-15)


def test_sk_vectorised_matches_blockwise_rules():
    s = lattice_water(4, seed=3)
    H0, S = model.build_h0_s(s, P)
    first, _, _ = model.ao_layout(s.species)
    pa, pb = model.atom_pairs_within(s.xyz, P["r_cut"])
    for a, b in list(zip(pa.tolist(), pb.tolist()))[::7]:
        R = s.xyz[b] - s.xyz[a]
        r = np.sqrt(model.dist2(np.zeros(3), R))
        d = np.exp(-r / P["r_decay"])
        Hb = model.sk_block(int(s.species[a]), int(s.species[b]), R, np.asarray(P["V0"]) * d)
        na, nb = Hb.shape
        assert np.allclose(H0[first[a]:first[a] + na, first[b]:first[b] + nb], Hb, rtol=0, atol=1e-15)


def test_h0_s_symmetric_and_s_positive_definite():
    s = lattice_water(16, seed=1)
    H0, S = model.build_h0_s(s, P)
    assert np.array_equal(H0, H0.T)
    assert np.array_equal(S, S.T)
    assert np.linalg.eigvalsh(S).min() > 0.5


def test_cutoff_inclusive():
    rc = P["r_cut"]
    H0, _ = model.build_h0_s(_pair(1, 1, [rc, 0.0, 0.0]), P)
    assert H0[0, 1] == pytest.approx(V(0, rc))
    H0, _ = model.build_h0_s(_pair(1, 1, [rc * (1 + 1e-12), 0.0, 0.0]), P)
    assert H0[0, 1] == 0.0


def _rotate_geometry(s, Rm):
    xyz = s.xyz @ Rm.T
    return WaterSystem(n_mol=s.n_mol, species=s.species, xyz=xyz, mol_of_atom=s.mol_of_atom,
                       site=s.site, group_of_mol=s.group_of_mol, n_groups=s.n_groups,
                       lattice_edge=s.lattice_edge)


def test_spectrum_rotation_invariant():
    s = lattice_water(3, seed=5)
    H0, S = model.build_h0_s(s, P)
    w0 = scipy.linalg.eigvalsh(H0, S)
    th = 0.7
    Rm = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    ax = 1.1
    Rx = np.array([[1, 0, 0], [0, np.cos(ax), -np.sin(ax)], [0, np.sin(ax), np.cos(ax)]])
    H1, S1 = model.build_h0_s(_rotate_geometry(s, Rx @ Rm), P)
    w1 = scipy.linalg.eigvalsh(H1, S1)
    assert np.allclose(w0, w1, atol=1e-12)


def test_gamma_limits():
    s = lattice_water(2, seed=0)
    G = model.gamma_matrix(s, P)
    U = np.where(s.species == 0, P["U_O"], P["U_H"])
    assert np.allclose(np.diag(G), U, rtol=1e-15)
    assert np.array_equal(G, G.T)
    far = _pair(0, 1, [1000.0, 0.0, 0.0])
    g = model.gamma_matrix(far, P)[0, 1]
    assert g == pytest.approx(1.0 / 1000.0, rel=1e-5)
    dq = np.linspace(-0.3, 0.4, s.n_atoms)
    assert np.allclose(model.gamma_times(s, P, dq, chunk=2), G @ dq, atol=1e-14)


def _energy_of_density(Pm, H0, S, G, atom_of_ao, q0, n_atoms):
    q = model.mulliken(Pm, S, atom_of_ao, n_atoms)
    dq = q - q0
    return model.energy(Pm, H0, dq, G @ dq)


def test_hamiltonian_is_energy_derivative():
    """dE/dP_mn = H_mn of Eq. (H_dftb2): a dropped 1/2 or a wrong atom index fails."""
    s = lattice_water(4, seed=2)
    H0, S = model.build_h0_s(s, P)
    G = model.gamma_matrix(s, P)
    _, atom_of_ao, n_ao = model.ao_layout(s.species)
    q0 = model.reference_population(s, P)
    rng = np.random.default_rng(0)
    w, C = scipy.linalg.eigh(H0, S)
    Pm = model.density(C[:, :4 * s.n_mol])
    Pm = Pm + 0.05 * (rng.standard_normal(Pm.shape) + rng.standard_normal(Pm.shape).T)
    q = model.mulliken(Pm, S, atom_of_ao, s.n_atoms)
    H = model.scc_hamiltonian(H0, S, G @ (q - q0), atom_of_ao)
    D = rng.standard_normal(Pm.shape)
    D = D + D.T
    h = 1e-5
    Ep = _energy_of_density(Pm + h * D, H0, S, G, atom_of_ao, q0, s.n_atoms)
    Em = _energy_of_density(Pm - h * D, H0, S, G, atom_of_ao, q0, s.n_atoms)
    assert (Ep - Em) / (2 * h) == pytest.approx(float((H * D).sum()), rel=1e-8)


def test_charges_sum_to_electron_count():
    s = lattice_water(5, seed=4)
    H0, S = model.build_h0_s(s, P)
    _, atom_of_ao, _ = model.ao_layout(s.species)
    w, C = scipy.linalg.eigh(H0, S)
    Pm = model.density(C[:, :4 * s.n_mol])
    q = model.mulliken(Pm, S, atom_of_ao, s.n_atoms)
    assert q.sum() == pytest.approx(8 * s.n_mol, rel=1e-13)
    dq = q - model.reference_population(s, P)
    assert dq.sum() == pytest.approx(0.0, abs=1e-12)


def test_sparse_and_dense_model_paths_agree():
    s = lattice_water(6, seed=6)
    H0, S = model.build_h0_s(s, P, dense=True)
    H0s, Ss = model.build_h0_s(s, P, dense=False)
    assert np.array_equal(H0s.toarray(), H0)
    _, atom_of_ao, _ = model.ao_layout(s.species)
    Q = np.linspace(-0.1, 0.1, s.n_atoms)
    assert np.allclose(model.scc_hamiltonian(H0s, Ss, Q, atom_of_ao).toarray(),
                       model.scc_hamiltonian(H0, S, Q, atom_of_ao), atol=1e-15)
    w, C = scipy.linalg.eigh(H0, S)
    Pm = model.density(C[:, :4 * s.n_mol])
    assert np.allclose(model.mulliken(Pm, Ss, atom_of_ao, s.n_atoms),
                       model.mulliken(Pm, S, atom_of_ao, s.n_atoms), atol=1e-13)


def test_dense_oracle_one_molecule_is_lowdin_eigensolve():
    """Single molecule: the SCC fixed point matches an independent Lowdin solve."""
    s = lattice_water(1, seed=0)
    r = dense.solve(s, P)
    assert r.converged
    H0, S = model.build_h0_s(s, P)
    _, atom_of_ao, _ = model.ao_layout(s.species)
    H = model.scc_hamiltonian(H0, S, r.Q, atom_of_ao)
    ws, Us = np.linalg.eigh(S)
    X = Us @ np.diag(ws ** -0.5) @ Us.T
    w = np.linalg.eigvalsh(X @ H @ X)
    assert np.allclose(w, r.eigenvalues, atol=1e-10)


def test_dense_oracle_self_consistency_and_idempotency():
    s = lattice_water(8, seed=0)
    r = dense.solve(s, P)
    assert r.converged
    H0, S = model.build_h0_s(s, P)
    _, atom_of_ao, _ = model.ao_layout(s.species)
    n_occ = 4 * s.n_mol
    # P S P = 2 P (P holds occupation 2), tr(PS) = N_e
    assert np.allclose(r.P @ S @ r.P, 2.0 * r.P, atol=1e-10)
    assert np.trace(r.P @ S) == pytest.approx(8 * s.n_mol, rel=1e-12)
    # the MOs solve H[dq] C = S C e with dq taken from those same MOs
    H = model.scc_hamiltonian(H0, S, model.gamma_matrix(s, P) @ r.dq, atom_of_ao)
    C = r.C[:, :n_occ]
    resid = H @ C - S @ C @ np.diag(r.eigenvalues[:n_occ])
    assert np.abs(resid).max() < 1e-7
    assert r.gap > 0.0
