"""FP64 CPU oracle for the sparse SCF of Scemama, Renon & Rapacioli (2014).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. It shares no code with the CUDA
library; both sides read the same seeded inputs from ``synth``.

Modules
-------
model       the synthetic SCC-DFTB model: Slater-Koster H0 and S, the SCC
            gamma, the Hamiltonian of Eq. (H_dftb)/(H_dftb2), Mulliken charges
            of Eq. (pop), the second-order energy.
dense       oracle A: the definition of the result, an SCC loop around a dense
            generalised eigensolve (the paper's LAPACK DSYGVD reference).
sparse      oracle B: the paper's sparse SCF algorithm (steps I-V) written out
            step by step on dense FP64 arrays holding explicit zeros.
adjoint     analytic SCC energy gradients (forces, Slater-Koster prefactors).
kmeans      the constrained k-means grouping of the molecules into MO groups.

Parity status: every function is pinned by tests in ``tests/test_oracle_*``;
none is "parity unpinned".
"""
