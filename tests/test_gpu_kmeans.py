"""GPU constrained k-means grouping (sscf_group_molecules) against the oracle.

The grouping is integer work decided by FP64 distance comparisons evaluated
without fused operations on both sides, so the groups, their number and the
iteration count must agree bit for bit: a cubic lattice, a thermally
displaced lattice, a strongly displaced (liquid-like) cluster and a ragged
count. The groups then drive a context on a displaced geometry, whose SCC
steps follow oracle B run with the same groups.
"""
import dataclasses

import numpy as np
import pytest

from gpu_common import P, context, library
from oracle import kmeans, sparse
from synth import lattice_water

pytestmark = pytest.mark.gpu

CASES = [(512, 0.0, 8), (1000, 0.3, 8), (300, 1.0, 8), (333, 0.2, 6)]


@pytest.mark.parametrize("n,sigma,n_link", CASES)
def test_groups_match_oracle_bit_for_bit(n, sigma, n_link):
    library()
    from paper_1402_2880_gb300 import group_molecules
    s = lattice_water(n, seed=1, displace_sigma_A=sigma)
    g, ng, it = group_molecules(s.xyz, n_link=n_link)
    rg, rng_, rit = kmeans.group_molecules(s.xyz, n_link=n_link)
    assert (ng, it) == (rng_, rit)
    assert np.array_equal(g, rg)
    assert np.bincount(g).max() <= n_link


def test_kmeans_groups_drive_the_scc():
    library()
    from paper_1402_2880_gb300 import group_molecules
    s = lattice_water(216, seed=2, displace_sigma_A=0.3)
    g, ng, _ = group_molecules(s.xyz, n_link=8)
    sg = dataclasses.replace(s, group_of_mol=g, n_groups=ng)
    ctx = context(sg)
    sc = sparse.SparseSCF(sg, P)
    assert ctx.n_groups == ng and np.array_equal(ctx.colouring(), sc.st.colour)
    eps = 1e-5
    ctx.set_thresholds(eps, 1e-4, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    ctx.reset_charges()
    st = sc.start(eps)
    assert np.abs(ctx.get_C() - st.C).max() < 1e-11
    for _ in range(2):
        info = ctx.step()
        ref = sc.step(st, eps)
        assert info["energy"] == pytest.approx(ref.energy, abs=1e-8 * s.n_atoms)
        assert info["n_rot"] == ref.n_rot
        q, _, _ = ctx.get_charges()
        assert np.abs(q - st.q_prev).max() < 1e-8
