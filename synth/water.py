"""Synthetic water-like clusters standing in for the paper's liquid-water boxes.

The paper benchmarks cubic boxes of liquid water (Section "Algorithm and
computational details"); neither its geometries nor its DFTB parameter
tables are available, so the workloads here are drawn from a seeded recipe:

* molecules sit on a simple cubic lattice of spacing 3.1 Angstrom
  (29.8 A^3 per molecule, close to liquid density); for a molecule count
  N the lattice edge is L = ceil(N^(1/3)) and the first N sites are used in
  x-fastest, then y, then z order; the cluster is open (no periodic images);
* each molecule has its oxygen on the site, O-H = 0.96 A, H-O-H = 104.5
  degrees, and a uniformly random orientation (normalised Gaussian
  quaternion drawn from numpy's PCG64 ``default_rng(seed)``);
* optional thermal displacements: every Cartesian atom component gets an
  independent N(0, sigma) shift from ``default_rng(displace_seed)``;
* MO groups are lattice cells of 2x2x2 sites, numbered in cell order
  (x fastest) with empty cells skipped; this partition stands in for the
  constrained k-means grouping of Section "Defining neighbouring lists".

Atoms are stored molecule-major (O, H1, H2); atomic orbitals per molecule are
O s, O px, O py, O pz, H1 s, H2 s. All lengths are returned in bohr.

This module draws inputs only; it contains none of the method's arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ANGSTROM_PER_BOHR = 0.529177210903  # CODATA 2018

SPECIES_O = 0
SPECIES_H = 1


@dataclasses.dataclass
class WaterSystem:
    n_mol: int
    species: np.ndarray        # (n_at,) int32, 0 = O (s,p: 4 AOs), 1 = H (s: 1 AO)
    xyz: np.ndarray            # (n_at, 3) float64, bohr
    mol_of_atom: np.ndarray    # (n_at,) int32
    site: np.ndarray           # (n_mol, 3) int32 lattice coordinates
    group_of_mol: np.ndarray   # (n_mol,) int32 MO-group index
    n_groups: int
    lattice_edge: int
    cluster_of_mol: np.ndarray | None = None   # batch of independent clusters, else None

    @property
    def n_atoms(self) -> int:
        return int(self.species.shape[0])

    @property
    def n_ao(self) -> int:
        return 6 * self.n_mol

    @property
    def n_occ(self) -> int:
        return 4 * self.n_mol

    @property
    def n_electrons(self) -> int:
        return 8 * self.n_mol


def default_params(**overrides) -> dict:
    """Synthetic Slater-Koster / SCC parameters of the water-like model.

    On-site energies, two-centre V(r) = V0 exp(-r / r_decay) for the
    ss-sigma, sp-sigma, pp-sigma and pp-pi integrals of H0 and (with S0) of
    S, the hard cut-off, the Hubbard parameters U of the SCC gamma, the
    reference populations and the SCF thresholds.
    """
    p = dict(
        onsite_O_s=-0.87,
        onsite_O_p=-0.33,
        onsite_H_s=-0.24,
        V0=(-0.50, 0.45, 0.40, -0.15),   # ss-sigma, sp-sigma, pp-sigma, pp-pi (Ha)
        S0=(0.45, -0.40, -0.35, 0.20),
        r_decay=1.6,                      # bohr
        r_cut=10.0,                       # bohr, pairs with r <= r_cut interact
        U_O=0.50,
        U_H=0.42,
        q0_O=6.0,
        q0_H=1.0,
        eps_mo=1e-6,                      # sparse threshold epsilon
        dq_tol=1e-5,                      # delta q_max criterion (10 eps)
        e_tol=1e-8,                       # energy change criterion (Ha)
        group_cut=20.0,                   # bohr, MO-group neighbour distance
        rot_cap_factor=10.0,              # rotations per sweep <= factor * N_occ
        mix_beta=0.2,
        max_scc=200,
    )
    p.update(overrides)
    return p


def _rotation_matrices(q: np.ndarray) -> np.ndarray:
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def lattice_water(n_mol: int, seed: int = 0, spacing_A: float = 3.1,
                  displace_sigma_A: float = 0.0, displace_seed: int = 5,
                  group_edge: int = 2) -> WaterSystem:
    """Seeded water-like cluster of ``n_mol`` molecules on a cubic lattice."""
    if n_mol < 1:
        raise ValueError("n_mol must be >= 1")
    L = 1
    while L * L * L < n_mol:
        L += 1
    idx = np.arange(n_mol)
    site = np.stack([idx % L, (idx // L) % L, idx // (L * L)], axis=1).astype(np.int32)

    rng = np.random.default_rng(seed)
    R = _rotation_matrices(rng.standard_normal((n_mol, 4)))
    d = 0.96
    half = math.radians(104.5) / 2.0
    frame = np.array([[0.0, 0.0, 0.0],
                      [d * math.cos(half), d * math.sin(half), 0.0],
                      [d * math.cos(half), -d * math.sin(half), 0.0]])
    xyz_A = site[:, None, :].astype(np.float64) * spacing_A + np.einsum("mij,kj->mki", R, frame)
    xyz_A = xyz_A.reshape(3 * n_mol, 3)
    if displace_sigma_A > 0.0:
        rng_d = np.random.default_rng(displace_seed)
        xyz_A = xyz_A + rng_d.normal(0.0, displace_sigma_A, size=xyz_A.shape)
    xyz = xyz_A / ANGSTROM_PER_BOHR

    species = np.tile(np.array([SPECIES_O, SPECIES_H, SPECIES_H], dtype=np.int32), n_mol)
    mol_of_atom = np.repeat(np.arange(n_mol, dtype=np.int32), 3)

    nc = (L + group_edge - 1) // group_edge
    cell = site // group_edge
    cell_id = cell[:, 0] + nc * (cell[:, 1] + nc * cell[:, 2])
    used = np.unique(cell_id)
    remap = -np.ones(nc ** 3, dtype=np.int64)
    remap[used] = np.arange(used.size)
    group_of_mol = remap[cell_id].astype(np.int32)
    return WaterSystem(n_mol=n_mol, species=species, xyz=np.ascontiguousarray(xyz),
                       mol_of_atom=mol_of_atom, site=site, group_of_mol=group_of_mol,
                       n_groups=int(used.size), lattice_edge=L)


def cluster_sizes(n_clusters: int = 256, lo: int = 200, hi: int = 3000, seed: int = 7) -> np.ndarray:
    """Molecule counts of the batched workload: uniform integers in [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, n_clusters)


def concat_clusters(systems) -> WaterSystem:
    """Independent clusters in one system: molecules, atoms and groups of
    cluster k follow those of cluster k-1, ``cluster_of_mol`` marks them.
    Coordinates are kept as drawn (clusters may overlap in space; nothing
    couples two clusters)."""
    species, xyz, mol_of_atom, site, groups, clusters = [], [], [], [], [], []
    m0 = g0 = 0
    for k, s in enumerate(systems):
        species.append(s.species)
        xyz.append(s.xyz)
        mol_of_atom.append(s.mol_of_atom + m0)
        site.append(s.site)
        groups.append(s.group_of_mol + g0)
        clusters.append(np.full(s.n_mol, k, dtype=np.int32))
        m0 += s.n_mol
        g0 += s.n_groups
    return WaterSystem(n_mol=m0, species=np.concatenate(species), xyz=np.concatenate(xyz),
                       mol_of_atom=np.concatenate(mol_of_atom).astype(np.int32), site=np.concatenate(site),
                       group_of_mol=np.concatenate(groups).astype(np.int32), n_groups=g0,
                       lattice_edge=max(s.lattice_edge for s in systems),
                       cluster_of_mol=np.concatenate(clusters))
