"""Stored reference values are the oracle's own (CPU).

tests/golden/config1_dense.json is written by tests/golden/make_config1_dense.py
from oracle A alone; this test recomputes it, so the file cannot go stale.
"""
import json
import os

import numpy as np

from oracle import dense
from synth import default_params, lattice_water

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_config1_dense_reference_is_the_oracles():
    with open(os.path.join(GOLDEN, "config1_dense.json")) as f:
        ref = json.load(f)
    s = lattice_water(32, seed=0)
    r = dense.solve(s, default_params(), dq_tol=1e-11, e_tol=1e-13)
    assert ref["converged"] and r.converged
    assert abs(r.energy - ref["energy"]) < 1e-11
    assert np.abs(r.q - np.asarray(ref["q"])).max() < 1e-10
