"""Helpers shared by the GPU parity tests (the CUDA path versus the oracle)."""
import functools

import numpy as np

from synth import default_params, lattice_water

P = default_params()


@functools.lru_cache(maxsize=None)
def library():
    from paper_1402_2880_gb300 import build, load
    build.build()
    return load()


def context(sysm, precision=0, **kw):
    library()
    from paper_1402_2880_gb300 import Context
    return Context.from_system(sysm, P, precision=precision, **kw)


@functools.lru_cache(maxsize=None)
def water(n, seed=0, sigma=0.0):
    return lattice_water(n, seed=seed, displace_sigma_A=sigma)


@functools.lru_cache(maxsize=None)
def oracle_scf(n, seed=0, sigma=0.0):
    from oracle import sparse
    return sparse.SparseSCF(water(n, seed, sigma), P)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
