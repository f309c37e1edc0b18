"""Writes config1_dense.json: the dense FP64 oracle's converged SCC state of
the 32-molecule cluster (4x4x2 water lattice, seed 0, default parameters).

Calls only ``oracle/`` (oracle A, the dense generalised eigensolve SCC) and
``synth/`` (the seeded geometry). The stored energy and Mulliken charges are
the reference that the benchmark's accuracy record and the tests compare the
GPU path's converged results with.

    python tests/golden/make_config1_dense.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense  # noqa: E402
from synth import default_params, lattice_water  # noqa: E402


def main():
    p = default_params()
    s = lattice_water(32, seed=0)
    r = dense.solve(s, p, dq_tol=1e-11, e_tol=1e-13)
    out = {"what": "oracle A (dense FP64 SCC, scipy eigh driver gvd): 32-molecule water lattice, seed 0, "
                   "default parameters, converged to dq 1e-11 e and 1e-13 Ha",
           "n_mol": 32, "n_atoms": int(s.n_atoms), "converged": bool(r.converged), "iterations": int(r.iterations),
           "energy": r.energy, "gap": r.gap, "q": [float(x) for x in r.q]}
    with open(os.path.join(HERE, "config1_dense.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
