"""Degenerate cluster sizes against the oracle: one molecule (one group with a
single self block), two and three molecules (one partial group), nine (a
full group plus a single molecule), and a batch of such clusters."""
import numpy as np
import pytest

from gpu_common import context, oracle_scf, water

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 3, 9])
def test_tiny_clusters_follow_oracle(n):
    s, sc, ctx = water(n), oracle_scf(n), context(water(n))
    eps = 1e-5
    ctx.set_thresholds(eps, 1e-4, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    ctx.reset_charges()
    st = sc.start(eps)
    assert np.abs(ctx.get_C() - st.C).max() < 1e-11
    for _ in range(3):
        info = ctx.step()
        ref = sc.step(st, eps)
        assert info["energy"] == pytest.approx(ref.energy, abs=1e-8 * s.n_atoms)
        assert info["n_rot"] == ref.n_rot
        q, _, _ = ctx.get_charges()
        assert np.abs(q - st.q_prev).max() < 1e-8
        assert np.abs(ctx.get_C() - st.C).max() < 1e-8


@pytest.mark.parametrize("prec,e_tol,q_tol", [(0, 1e-8, 1e-9), (1, 1e-6, 1e-3)])
def test_tiny_batch_equals_clusters_alone(prec, e_tol, q_tol):
    from synth import concat_clusters, lattice_water
    parts = [lattice_water(n, seed=k) for k, n in enumerate([1, 2, 5, 9])]
    eps = 1e-5

    def prep(c):
        c.set_thresholds(eps, 10 * eps, 1e-8)
        c.guess()
        c.orthonormalise(0)
        c.reset_charges()
        return c

    cb = prep(context(concat_clusters(parts), precision=prec))
    singles = [prep(context(part, precision=prec)) for part in parts]
    a0 = np.cumsum([0] + [3 * part.n_mol for part in parts])
    for step in range(3):
        cb.step()
        Eb, _ = cb.cluster_results()
        qb, _, _ = cb.get_charges()
        for k, c in enumerate(singles):
            info = c.step()
            assert Eb[k] == pytest.approx(info["energy"], abs=e_tol * parts[k].n_atoms), (step, k)
            q, _, _ = c.get_charges()
            assert np.abs(qb[a0[k]:a0[k + 1]] - q).max() < q_tol
