"""Batch mode: several independent clusters in one context behave exactly as
each cluster alone (same structure, guess, orthonormalisation, SCC steps,
per-cluster energies and charges), with one set of kernel launches."""
import numpy as np
import pytest

from gpu_common import P, context
from synth import concat_clusters, lattice_water

pytestmark = pytest.mark.gpu


def _prep(ctx, eps):
    ctx.set_thresholds(eps, 10 * eps, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    ctx.reset_charges()


def test_batch_equals_separate_clusters():
    parts = [lattice_water(8, seed=1), lattice_water(20, seed=2), lattice_water(32, seed=3)]
    batch = concat_clusters(parts)
    eps = 1e-5
    cb = context(batch)
    _prep(cb, eps)
    singles = [context(s) for s in parts]
    for c in singles:
        _prep(c, eps)
    a0 = np.cumsum([0] + [3 * s.n_mol for s in parts])
    for step in range(3):
        cb.step()
        Eb, dqb = cb.cluster_results()
        qb, _, _ = cb.get_charges()
        for k, c in enumerate(singles):
            info = c.step()
            E, dq = c.cluster_results()
            assert E[0] == pytest.approx(info["energy"], abs=1e-9)
            assert Eb[k] == pytest.approx(E[0], abs=1e-8), (step, k)
            assert dqb[k] == pytest.approx(dq[0], abs=1e-9)
            q, _, _ = c.get_charges()
            assert np.abs(qb[a0[k]:a0[k + 1]] - q).max() < 1e-9
    assert cb.n_groups == sum(s.n_groups for s in parts)


def test_batch_run_converges_every_cluster():
    parts = [lattice_water(8, seed=4), lattice_water(16, seed=5)]
    batch = concat_clusters(parts)
    cb = context(batch)
    out = cb.run()
    assert out["converged"]
    E, dq = cb.cluster_results()
    for k, s in enumerate(parts):
        c = context(s)
        o = c.run()
        assert abs(E[k] - o["energy"]) < 1e-6 * s.n_mol * 3


@pytest.mark.parametrize("prec,e_tol,q_tol", [(0, 1e-10, 1e-9), (1, 1e-6, 1e-3)])
def test_batch_of_drawn_cluster_sizes_equals_separate_clusters(prec, e_tol, q_tol):
    """Three clusters of the batched workload's seed-7 size draw (214, 355 and 830
    molecules): the batch reproduces each cluster alone. In FP64 the only
    difference is the summation order of the gamma tiles (the batch starts them
    at other atoms); in mixed precision those FP32 tile sums differ by FP32
    rounding, which can flip a pair at the rotation cap. At these clusters' small
    SCC gaps (~0.01 Ha) one flipped rotation moves charges by ~1e-4 e, so mixed
    runs are compared to 1e-6 Ha/atom in energy and 1e-3 e in charge."""
    from synth import cluster_sizes
    sizes = cluster_sizes()
    picks = [13, 8, 7]
    assert [int(sizes[k]) for k in picks] == [214, 355, 830]
    parts = [lattice_water(int(sizes[k]), seed=k) for k in picks]
    eps = 1e-5
    cb = context(concat_clusters(parts), precision=prec)
    _prep(cb, eps)
    singles = [context(s, precision=prec) for s in parts]
    for c in singles:
        _prep(c, eps)
    a0 = np.cumsum([0] + [3 * s.n_mol for s in parts])
    for step in range(2):
        cb.step()
        Eb, _ = cb.cluster_results()
        qb, _, _ = cb.get_charges()
        for k, c in enumerate(singles):
            info = c.step()
            assert abs(Eb[k] - info["energy"]) < e_tol * 3 * parts[k].n_mol, (step, k)
            q, _, _ = c.get_charges()
            assert np.abs(qb[a0[k]:a0[k + 1]] - q).max() < q_tol, (step, k)
