"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws geometries and fixes model parameters. It holds none of
the sparse-SCF arithmetic: no matrix elements, no charges, no energies.
"""
from .water import (  # noqa: F401
    ANGSTROM_PER_BOHR,
    WaterSystem,
    default_params,
    lattice_water,
    cluster_sizes,
    concat_clusters,
)
