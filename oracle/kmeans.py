"""Constrained k-means grouping of molecules into MO groups (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section "Defining neighbouring lists of atoms and MOs": a set of centres is
spread evenly over space; every unit is linked to its closest centre, except
that a centre takes no more than N_link units (a unit that finds its closest
centre full goes to the next closest with room); every centre then moves to
the centroid of its units; this repeats until the average displacement of
the centres falls below a threshold or a number of iterations (typically
100) is reached.

Readings (the GPU library implements the same ones):

* The unit is a molecule, at its first (oxygen) atom, because the MO groups
  of this library are sets of whole molecules (at most 8 per group).
* "Spread evenly": a grid of g_x x g_y x g_z centres over the bounding box of
  the molecules, cell centres at lo + (2 i + 1) L / (2 g). Starting from
  1 x 1 x 1, the axis with the largest L / g (lowest axis on ties) is refined
  until there are at least ceil(N / N_link) centres; extents below 1 bohr
  count as 1 bohr.
* "Closest centre with room": the paper's attribution depends on the order in
  which units are visited and is evened out by shuffling the centres each
  iteration. Here it is the molecule-proposing deferred-acceptance matching:
  molecules propose to centres in increasing (distance^2, centre index); a
  centre keeps the N_link proposals with the smallest (distance^2, molecule
  index) and rejects the rest, who propose to their next centre. Its result
  is unique and independent of any visiting order (stable: no molecule and
  centre would both rather be linked to each other), so no shuffle is needed.
* Centroid: the members' coordinates summed in increasing molecule index,
  divided by their count; a centre without members stays where it is.
* Average displacement: the Euclidean moves of all centres summed in centre
  order, divided by the number of centres.
* Groups: the centres that hold molecules, numbered in centre order.

Squared distances are (dx*dx + dy*dy) + dz*dz with no fused operations, on
both sides, so every comparison is bit-identical.
"""
from __future__ import annotations

import math

import numpy as np


def initial_centres(pos: np.ndarray, n_link: int) -> np.ndarray:
    """Grid of centres over the bounding box (see the module notes)."""
    lo = pos.min(axis=0)
    hi = pos.max(axis=0)
    L = [max(float(hi[d] - lo[d]), 1.0) for d in range(3)]
    need = -(-pos.shape[0] // n_link)
    g = [1, 1, 1]
    while g[0] * g[1] * g[2] < need:
        ratio = [L[d] / g[d] for d in range(3)]
        g[ratio.index(max(ratio))] += 1
    out = []
    for k in range(g[2]):
        for j in range(g[1]):
            for i in range(g[0]):
                idx = (i, j, k)
                out.append([float(lo[d]) + ((2 * idx[d] + 1) * L[d]) / (2 * g[d]) for d in range(3)])
    return np.array(out)


def dist2(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    d = b - a
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def attribute(pos: np.ndarray, centres: np.ndarray, n_link: int) -> np.ndarray:
    """Deferred acceptance: the centre of every molecule, at most n_link per centre."""
    n, nc = pos.shape[0], centres.shape[0]
    D = dist2(pos[:, None, :], centres[None, :, :])                  # (n, nc)
    pref = np.lexsort((np.broadcast_to(np.arange(nc), D.shape), D), axis=1)   # by (d2, centre)
    nxt = np.zeros(n, dtype=np.int64)                                # next preference to try
    holder = -np.ones(n, dtype=np.int64)
    while True:
        free = np.nonzero(holder < 0)[0]
        if free.size == 0:
            return holder
        prop = pref[free, nxt[free]]
        nxt[free] += 1
        changed = set(prop.tolist())
        for c in sorted(changed):
            cand = np.concatenate([np.nonzero(holder == c)[0], free[prop == c]])
            order = np.lexsort((cand, D[cand, c]))                     # by (d2, molecule)
            keep = cand[order[:n_link]]
            drop = cand[order[n_link:]]
            holder[keep] = c
            holder[drop] = -1


def centroids(pos: np.ndarray, holder: np.ndarray, centres: np.ndarray) -> np.ndarray:
    new = centres.copy()
    for c in range(centres.shape[0]):
        members = np.nonzero(holder == c)[0]                          # increasing molecule index
        if members.size == 0:
            continue
        s = [0.0, 0.0, 0.0]
        for m in members.tolist():
            for d in range(3):
                s[d] += float(pos[m, d])
        new[c] = [s[d] / members.size for d in range(3)]
    return new


def group_molecules(xyz: np.ndarray, n_link: int = 8, max_iter: int = 100, tol: float = 1e-3):
    """(group_of_mol, n_groups, iterations) of a system with atoms O, H, H per molecule."""
    pos = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)[0::3]
    centres = initial_centres(pos, n_link)
    holder = attribute(pos, centres, n_link)
    it = 0
    for it in range(1, max_iter + 1):
        new = centroids(pos, holder, centres)
        moved = 0.0
        for c in range(centres.shape[0]):
            d = new[c] - centres[c]
            moved += math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
        centres = new
        holder = attribute(pos, centres, n_link)
        if moved / centres.shape[0] < tol:
            break
    used = np.unique(holder)
    remap = -np.ones(centres.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return remap[holder].astype(np.int32), int(used.size), it
