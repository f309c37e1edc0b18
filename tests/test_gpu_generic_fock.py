"""A caller-built Fock matrix through the same C^T X C and rotation machinery.

Only step IV of the paper's algorithm (the Hamiltonian build) is specific to
DFTB; an HF-type method builds its own Fock matrix X from the density matrix
and hands it to steps V and III. sscf_set_fock_blocks takes such an X on the
molecule-pair pattern and sscf_get_density_blocks returns P = 2 C_occ C_occ^T
on the same pattern. Both are checked against the FP64 oracle on a random
symmetric X (100 molecules, ragged groups): the transform and the sweep
element by element, the pair list bit for bit, P to FP64 rounding.
"""
import numpy as np
import pytest

from gpu_common import P, context, oracle_scf, water
from oracle import sparse

pytestmark = pytest.mark.gpu


def _dense(mn, blocks, n_ao):
    M = np.zeros((n_ao, n_ao))
    for (m, n), b in zip(mn, blocks):
        M[6 * m:6 * m + 6, 6 * n:6 * n + 6] = b
    return M


def test_caller_fock_transform_sweep_and_density():
    n, eps = 100, 1e-5
    s, sc = water(n), oracle_scf(n)
    ctx = context(s)
    ctx.set_thresholds(eps, 10 * eps, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    C0 = ctx.get_C()
    mn, _, H0b, _ = ctx.get_blocks()
    rng = np.random.default_rng(21)
    idx = {(int(m), int(k)): e for e, (m, k) in enumerate(mn)}
    X = np.empty((len(mn), 6, 6))
    for e, (m, k) in enumerate(mn):
        if m < k:
            X[e] = H0b[e] + 0.05 * rng.standard_normal((6, 6))
            X[idx[(int(k), int(m))]] = X[e].T
        elif m == k:
            a = H0b[e] + 0.05 * rng.standard_normal((6, 6))
            X[e] = 0.5 * (a + a.T)
    ctx.set_fock_blocks(X)
    Xd = _dense(mn, X, s.n_ao)
    off = ~np.eye(s.n_ao, dtype=bool)
    Xd[off & (np.abs(Xd) < eps)] = 0.0          # the same threshold as the DFTB build
    n_rot, _ = ctx.rotate_sweep()
    F, Fd = ctx.get_F()
    F_ref, Fd_ref, mask = sparse.transform_ov(C0, Xd, sc.st)
    assert np.abs(F - F_ref).max() <= 1e-12 * max(np.abs(F_ref).max(), 1.0)
    assert np.abs(Fd - Fd_ref).max() <= 1e-12 * max(np.abs(Fd_ref).max(), 1.0)
    sel = sparse.select_pairs(F, mask, eps, int(P["rot_cap_factor"] * sc.st.n_occ))
    assert n_rot == int(sel.sum()) and n_rot > 0
    _, _, i, j = ctx.pairs()
    got = np.zeros_like(sel)
    got[i, j - sc.st.n_occ] = True
    assert np.array_equal(got, sel)
    ref = C0.copy()
    sparse.rotate_sweep(ref, F, Fd, sc.st, sel, eps)
    C = ctx.get_C()
    assert np.abs(C - ref).max() < 1e-11
    # P on the pattern, for the caller's next Fock build
    Pb = ctx.density_blocks()
    Co = C[:, :sc.st.n_occ]
    Pref = 2.0 * Co @ Co.T
    for e, (m, k) in enumerate(mn):
        blk = Pref[6 * m:6 * m + 6, 6 * k:6 * k + 6]
        assert np.abs(Pb[e] - blk).max() <= 1e-12 * max(np.abs(Pref).max(), 1.0)
    # the charges and the mixing state are untouched by the density read-out
    q0, dq0, Q0 = ctx.get_charges()
    ctx.density_blocks()
    q1, dq1, Q1 = ctx.get_charges()
    assert np.array_equal(q0, q1) and np.array_equal(dq0, dq1) and np.array_equal(Q0, Q1)


def test_caller_fock_rejects_nonfinite():
    from paper_1402_2880_gb300 import SscfError
    s = water(32)
    ctx = context(s)
    mn, _, H0b, _ = ctx.get_blocks()
    X = H0b.copy()
    X[3, 1, 2] = np.nan
    with pytest.raises(SscfError) as e:
        ctx.set_fock_blocks(X)
    assert e.value.status == -4
