"""Pins of the oracle's analytic gradients (the adjoint of the SCC energy).

* the Slater-Koster derivative blocks against central differences of the blocks;
* W = 1/2 P H P against sum_i n_i e_i c_i c_i^T from the dense eigensolve;
* forces and the 8 parameter gradients against central finite differences of
  the converged dense SCC energy (h = 1e-4 bohr, 1e-5 Ha), relative to the
  largest gradient component, with no atom pair within 2h of the cut-off.
"""
import numpy as np
import pytest

from oracle import adjoint, dense, model
from synth import default_params, lattice_water
from synth.water import WaterSystem

P = default_params()


@pytest.mark.parametrize("sa,sb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_sk_block_grad_matches_finite_difference(sa, sb):
    rng = np.random.default_rng(sa * 2 + sb)
    V0 = np.asarray(P["V0"])
    for _ in range(5):
        R = rng.normal(0, 2.5, 3)
        g = adjoint.sk_block_grad(sa, sb, R, V0, P["r_decay"])
        h = 1e-6
        for k in range(3):
            dR = np.zeros(3)
            dR[k] = h

            def blk(RR):
                r = np.sqrt(model.dist2(np.zeros(3), RR))
                return model.sk_block(sa, sb, RR, V0 * np.exp(-r / P["r_decay"]))
            fd = (blk(R + dR) - blk(R - dR)) / (2 * h)
            assert np.allclose(g[k], fd, atol=1e-8)


def _converged(s, p):
    return dense.solve(s, p, dq_tol=1e-12, e_tol=1e-14, max_iter=3000)


def test_energy_weighted_density_identity():
    s = lattice_water(4, seed=1)
    r = _converged(s, P)
    H0, S = model.build_h0_s(s, P)
    _, atom_of_ao, _ = model.ao_layout(s.species)
    H = model.scc_hamiltonian(H0, S, model.gamma_matrix(s, P) @ r.dq, atom_of_ao)
    n_occ = 4 * s.n_mol
    C = r.C[:, :n_occ]
    W_can = 2.0 * C @ np.diag(r.eigenvalues[:n_occ]) @ C.T
    assert np.abs(adjoint.energy_weighted_density(r.P, H) - W_can).max() < 1e-9


def _shift(s, atom, k, h):
    xyz = s.xyz.copy()
    xyz[atom, k] += h
    return WaterSystem(n_mol=s.n_mol, species=s.species, xyz=xyz, mol_of_atom=s.mol_of_atom, site=s.site,
                       group_of_mol=s.group_of_mol, n_groups=s.n_groups, lattice_edge=s.lattice_edge)


def _margin_ok(s, atom, h, rc):
    d = np.sqrt(((s.xyz - s.xyz[atom]) ** 2).sum(1))
    return not np.any(np.abs(d - rc) < 4 * h)


@pytest.mark.slow
def test_gradients_match_finite_differences():
    s = lattice_water(8, seed=2, displace_sigma_A=0.1)
    r = _converged(s, P)
    g, gp = adjoint.gradients(s, P, r.P, r.dq)
    h = 1e-4
    scale = np.abs(g).max()
    rng = np.random.default_rng(0)
    checked = 0
    for atom in rng.permutation(s.n_atoms):
        if checked >= 6:
            break
        if not _margin_ok(s, atom, h, P["r_cut"]):
            continue
        for k in range(3):
            ep = _converged(_shift(s, atom, k, h), P).energy
            em = _converged(_shift(s, atom, k, -h), P).energy
            assert abs((ep - em) / (2 * h) - g[atom, k]) < 1e-7 * scale
        checked += 1
    assert checked >= 4
    hp = 1e-5
    pscale = np.abs(gp).max()
    for j in range(8):
        key, idx = ("V0", j) if j < 4 else ("S0", j - 4)
        vp = list(P[key])
        vm = list(P[key])
        vp[idx] += hp
        vm[idx] -= hp
        ep = _converged(s, dict(P, **{key: tuple(vp)})).energy
        em = _converged(s, dict(P, **{key: tuple(vm)})).energy
        assert abs((ep - em) / (2 * hp) - gp[j]) < 1e-5 * pscale
