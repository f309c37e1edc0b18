"""Pins of the oracle's constrained k-means grouping (CPU).

Section "Defining neighbouring lists of atoms and MOs": units linked to their
closest centre with room (at most N_link per centre), centres moved to the
centroids of their units, repeated to convergence. Checked against facts that
do not depend on the implementation:

* the links are a stable matching (no molecule and centre would both rather
  be linked to each other), every molecule is linked and no centre holds more
  than N_link molecules;
* the links do not depend on the order of the molecules (a relabelling gives
  the same partition), the property that lets the paper's shuffle go;
* the centroid step is the arithmetic mean of the members;
* the starting grid holds at least ceil(N / N_link) centres inside the
  bounding box, a full cube for a cubic lattice;
* on the 8x8x8 water lattice with N_link = 8 the grouping ends with 64 full
  groups of neighbouring molecules.
"""
import numpy as np

from oracle import kmeans
from synth import lattice_water


def _pos(n, sigma=0.0, seed=0):
    s = lattice_water(n, seed=seed, displace_sigma_A=sigma)
    return s, s.xyz[0::3]


def test_links_are_a_stable_matching_within_capacity():
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 40.0, size=(200, 3))
    cen = kmeans.initial_centres(pos, 8)
    h = kmeans.attribute(pos, cen, 8)
    assert np.all(h >= 0)
    counts = np.bincount(h, minlength=cen.shape[0])
    assert counts.max() <= 8
    D = kmeans.dist2(pos[:, None, :], cen[None, :, :])
    for m in range(pos.shape[0]):
        cm = h[m]
        for c in range(cen.shape[0]):
            if (D[m, c], c) >= (D[m, cm], cm):
                continue
            # m prefers c: c must be full of molecules it prefers to m
            members = np.nonzero(h == c)[0]
            assert members.size == 8
            assert all((D[k, c], k) < (D[m, c], m) for k in members)


def test_links_do_not_depend_on_the_molecule_order():
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, 30.0, size=(150, 3))
    cen = kmeans.initial_centres(pos, 8)
    h = kmeans.attribute(pos, cen, 8)
    perm = rng.permutation(pos.shape[0])
    hp = kmeans.attribute(pos[perm], cen, 8)
    back = np.empty_like(hp)
    back[perm] = hp
    assert np.array_equal(back, h)


def test_centroids_are_member_means():
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 20.0, size=(90, 3))
    cen = kmeans.initial_centres(pos, 6)
    h = kmeans.attribute(pos, cen, 6)
    new = kmeans.centroids(pos, h, cen)
    for c in range(cen.shape[0]):
        m = h == c
        want = pos[m].mean(axis=0) if m.any() else cen[c]
        assert np.allclose(new[c], want, rtol=0, atol=1e-12)


def test_initial_grid():
    s, pos = _pos(512)
    cen = kmeans.initial_centres(pos, 8)
    assert cen.shape[0] == 64                       # 4 x 4 x 4 for the 8 x 8 x 8 lattice
    lo, hi = pos.min(axis=0), pos.max(axis=0)
    assert np.all(cen >= lo) and np.all(cen <= hi)
    _, pos2 = _pos(100, sigma=0.3)
    cen2 = kmeans.initial_centres(pos2, 8)
    assert cen2.shape[0] >= 13


def test_lattice_grouping_is_full_and_local():
    s, pos = _pos(512)
    g, ng, it = kmeans.group_molecules(s.xyz, n_link=8)
    assert ng == 64 and it >= 1
    assert np.all(np.bincount(g) == 8)
    spacing = 3.1 / 0.529177210903
    for k in range(ng):
        p = pos[g == k]
        span = (p.max(axis=0) - p.min(axis=0)).max()
        assert span < 3.5 * spacing                 # neighbouring molecules, not scattered ones
