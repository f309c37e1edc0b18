"""Mixed precision (FP32 storage and sweeps, FP64 angles, norms and sums)
against the FP64 oracle, element by element.

The kernels the benchmark times run in FP32 storage: the C^T H C transform,
the rotation sweep (register-resident kernel on blocks between full groups,
generic kernel elsewhere) and the occupied orthonormalisation pass. Each is
fed the same inputs as the oracle (the FP32 MOs widened to FP64, and the
GPU's own F or sigma where a decision depends on them) and compared element
by element:

* F = C^T H C within 1024 u times the sum of the absolute terms
  (|C|^T |H| |C|, u = 2^-24): H, Y = H C and F are rounded to FP32 once
  each, a value of Y sums 6 terms per pattern neighbour in FP32 (at most a
  few hundred), and F sums at most 32 row blocks (192 terms) in FP32 between
  FP64 flushes, so the worst case stays below 1024 u;
* the sweeps within the forward error bound of ``fp32_bounds`` (every FP32
  rounding of every update, truncation decisions that may differ only where
  a value lies within that bound of the threshold);
* pair lists bit for bit (they are decided on the GPU's own F and sigma).

Sizes: 100 molecules (ragged groups: both sweep kernels in one colour) and
216 molecules (all groups full: the register-resident kernels throughout).
The converged comparison (config 1, 32 molecules) checks the accuracy
targets of the mixed path against both oracles: |dE| <= 1e-6 Ha/atom,
charges within 1e-5 e.
"""
import numpy as np
import pytest

import fp32_bounds
from gpu_common import P, context, oracle_scf, water
from oracle import dense, sparse

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
MIXED = 1


def _prepared_mixed(n, eps):
    s, sc = water(n), oracle_scf(n)
    ctx = context(s, precision=MIXED)
    ctx.set_thresholds(eps, 10 * eps, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    return s, sc, ctx, ctx.get_C()


@pytest.mark.parametrize("n", [100, 216])
def test_mixed_transform_and_rotation_sweep_elementwise(n):
    eps = 1e-5
    s, sc, ctx, C0 = _prepared_mixed(n, eps)
    st = sc.st
    rng = np.random.default_rng(n + 1)
    Q = rng.normal(0.0, 0.05, s.n_atoms)
    ctx.set_charges(Q_in=Q)
    ctx.build_fock()
    n_rot, _ = ctx.rotate_sweep()
    F, Fd = ctx.get_F()
    # the transform: FP64 oracle on the widened FP32 MOs
    H = sparse.fock(sc.H0, sc.S, Q, sc.atom_of_ao, eps)
    F_ref, Fd_ref, mask = sparse.transform_ov(C0, H, st)
    absC, absH = np.abs(C0), np.abs(H)
    terms = absC.T @ (absH @ absC)
    no = st.n_occ
    assert np.all(np.abs(F - F_ref) <= 1024 * U * np.where(mask, terms[:no, no:], 0.0))
    assert np.all(np.abs(Fd - Fd_ref) <= 1024 * U * np.diag(terms))
    assert np.all(F[~mask] == 0)
    # the selection on the GPU's own F: bit-exact
    k_max = int(P["rot_cap_factor"] * no)
    sel = sparse.select_pairs(F, mask, eps, k_max)
    assert n_rot == int(sel.sum())
    _, _, i, j = ctx.pairs()
    got = np.zeros_like(sel)
    got[i, j - no] = True
    assert np.array_equal(got, sel)
    # the FP32 sweep against the FP64 oracle sweep on the same F
    ref = C0.copy()
    sparse.rotate_sweep(ref, F, Fd, st, sel, eps)
    vals, bound = fp32_bounds.rotations(C0, F, Fd, st, sel, eps)
    assert np.array_equal(vals, ref)
    C = ctx.get_C()
    err = np.abs(C - ref)
    assert np.all(err <= bound), f"worst excess {np.max(err - bound):.3e}"
    # the bound means something: a few FP32 units on the values that matter
    big = np.abs(ref) > 1e-3
    assert np.median(bound[big] / np.abs(ref[big])) < 1e-5


@pytest.mark.parametrize("n", [100, 216])
def test_mixed_occupied_pass_elementwise(n):
    eps = 1e-4
    s, sc, ctx, C0 = _prepared_mixed(n, eps)
    st = sc.st
    rng = np.random.default_rng(7)
    C1 = C0.copy()
    no = st.n_occ
    C1[:, :no] += 1e-3 * rng.standard_normal(C1[:, :no].shape) * (C1[:, :no] != 0)
    ctx.set_C(C1)
    C1 = ctx.get_C()                       # as stored: FP32
    passes, eta = ctx.orthonormalise(1, max_pass=1)
    sigma = ctx.get_overlap()
    assert sigma.shape == (no, no)
    # the GPU's overlaps against the FP64 product on the same MOs
    mos = np.arange(no)
    mask = sparse.overlap_mask(st, mos)
    sig_ref = np.where(mask, C1[:, mos].T @ (sc.S @ C1[:, mos]), 0.0)
    terms = np.abs(C1[:, mos]).T @ (np.abs(sc.S) @ np.abs(C1[:, mos]))
    assert np.all(np.abs(sigma - sig_ref) <= 1024 * U * np.where(mask, terms, 0.0))
    tol = max(eps / 100, 2.0 ** -19)
    ref = C1.copy()
    reta, ncombo = sparse.ortho_pass(ref, sc.S, st, "occ", tol, 1e-3 * eps, sigma=sigma)
    assert eta == reta
    _, _, i, j = ctx.pairs()
    assert ncombo == i.size
    vals, bound = fp32_bounds.combinations(C1, sigma, st, "occ", tol, 1e-3 * eps)
    assert np.array_equal(vals, ref)
    C = ctx.get_C()
    err = np.abs(C - ref)
    assert np.all(err <= bound), f"worst excess {np.max(err - bound):.3e}"
    big = np.abs(ref) > 1e-3
    assert np.median(bound[big] / np.abs(ref[big])) < 1e-3


def test_run_config1_mixed_converges_to_both_oracles():
    """Config 1 converged tightly (charges to 1e-7 e, energy to 1e-10 Ha, so
    that the SCF criterion itself stays below the tolerances).

    Energy within 1e-6 Ha/atom of oracle B (the sparse method in FP64, same
    eps) and of oracle A (the dense eigensolve, stored by
    tests/golden/make_config1_dense.py). Charges: at eps = 1e-6 the sparse
    method itself lands 1.2e-5 e from the dense charges (couplings below eps
    are never rotated), and two converged sparse solutions whose rotation
    decisions differ near eps (FP32 against FP64 values of F) differ by that
    much too: within max(1e-5, that method error) of oracle B, and within the
    method error plus 1e-5 e of oracle A."""
    import json
    import os

    from paper_1402_2880_gb300 import Context
    from synth import default_params
    pt = default_params(dq_tol=1e-7, e_tol=1e-10)
    s = water(32)
    ctx = Context.from_system(s, pt, precision=MIXED)
    out = ctx.run()
    assert out["converged"]
    q, _, _ = ctx.get_charges()
    ref_b = sparse.SparseSCF(s, pt).run()
    assert ref_b["converged"]
    with open(os.path.join(os.path.dirname(__file__), "golden", "config1_dense.json")) as f:
        ref_a = json.load(f)
    qa = np.asarray(ref_a["q"])
    method = float(np.abs(ref_b["q"] - qa).max())
    print(f"vs B: |dE|/atom {abs(out['energy'] - ref_b['energy']) / s.n_atoms:.3e}, "
          f"max|dq| {np.abs(q - ref_b['q']).max():.3e}; vs A: |dE|/atom "
          f"{abs(out['energy'] - ref_a['energy']) / s.n_atoms:.3e}, max|dq| {np.abs(q - qa).max():.3e} "
          f"(B vs A {method:.3e})")
    assert abs(out["energy"] - ref_b["energy"]) / s.n_atoms <= 1e-6
    assert np.abs(q - ref_b["q"]).max() <= max(1e-5, method)
    assert abs(out["energy"] - ref_a["energy"]) / s.n_atoms <= 1e-6
    assert np.abs(q - qa).max() <= method + 1e-5


def test_set_precision_keeps_the_mos():
    s = water(32)
    ctx = context(s, precision=MIXED)
    ctx.set_thresholds(1e-5, 1e-4, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    C32 = ctx.get_C()
    E32 = ctx.reset_charges()
    ctx.set_precision(0)
    assert np.array_equal(ctx.get_C(), C32)           # widening is exact
    E64 = ctx.reset_charges()
    assert abs(E64 - E32) / s.n_atoms < 1e-6          # FP64 sums of the same MOs
    C64 = C32 + 1e-9 * (C32 != 0)
    ctx.set_C(C64)
    ctx.set_precision(MIXED)
    assert np.array_equal(ctx.get_C(), C64.astype(np.float32).astype(np.float64))
    ctx.step()                                        # the narrowed context still steps
