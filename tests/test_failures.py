"""Failure handling made on the host (no GPU fault is ever provoked).

CPU: invalid layouts, non-finite coordinates and unknown parameters are refused
before any CUDA call; an allocator hook that refuses memory gives SSCF_ERR_OOM. GPU: a row
capacity that is too small gives SSCF_ERR_CAPACITY and leaves C and the
charges as they were.
"""
import ctypes

import numpy as np
import pytest

from synth import default_params, lattice_water

P = default_params()


def _lib():
    from paper_1402_2880_gb300 import _lib, build
    build.build()
    return _lib


def test_nonfinite_coordinates_refused():
    _lib_ = _lib()
    s = lattice_water(4)
    xyz = s.xyz.copy()
    xyz[3, 1] = np.nan
    with pytest.raises(_lib_.SscfError) as e:
        _lib_.Context(s.species, xyz, s.group_of_mol, P)
    assert e.value.status == -4


def test_oversized_group_refused():
    _lib_ = _lib()
    s = lattice_water(16)
    with pytest.raises(_lib_.SscfError) as e:
        _lib_.Context(s.species, s.xyz, np.zeros(s.n_mol, dtype=np.int32), P)   # 16 molecules in one group
    assert e.value.status == -1


def test_cluster_order_refused():
    _lib_ = _lib()
    s = lattice_water(8)
    cl = np.array([0, 1, 0, 1, 0, 1, 0, 1], dtype=np.int32)
    with pytest.raises(_lib_.SscfError) as e:
        _lib_.Context(s.species, s.xyz, s.group_of_mol, P, cluster_of_mol=cl)
    assert e.value.status == -1


def test_unknown_sweep_variant_refused():
    _lib_ = _lib()
    s = lattice_water(8)
    for v in (-1, 3):
        with pytest.raises(_lib_.SscfError) as e:
            _lib_.Context(s.species, s.xyz, s.group_of_mol, P, apply_variant=v)
        assert e.value.status == -1


def test_allocator_failure_reports_oom():
    _lib_ = _lib()
    lib = _lib_.load()
    calls = []

    @_lib_.ALLOC_FN
    def refuse(nbytes, user):
        calls.append(nbytes)
        return None

    @_lib_.FREE_FN
    def release(ptr, user):
        raise AssertionError("nothing was allocated")

    assert lib.sscf_set_allocator(refuse, release, None) == 0
    try:
        s = lattice_water(4)
        with pytest.raises(_lib_.SscfError) as e:
            _lib_.Context(s.species, s.xyz, s.group_of_mol, P)
        assert e.value.status == -2
        assert len(calls) == 1
    finally:
        assert lib.sscf_set_allocator(ctypes.cast(None, _lib_.ALLOC_FN), ctypes.cast(None, _lib_.FREE_FN), None) == 0


@pytest.mark.gpu
def test_capacity_overflow_keeps_state():
    from gpu_common import context, water
    from paper_1402_2880_gb300 import SscfError
    ctx = context(water(100), cap_tiles=3)
    ctx.set_thresholds(1e-5, 1e-4, 1e-8)
    ctx.guess()
    C0 = ctx.get_C()
    q0, dq0, Q0 = ctx.get_charges()
    with pytest.raises(SscfError) as e:
        ctx.orthonormalise(0)
    assert e.value.status == -5
    assert np.array_equal(ctx.get_C(), C0)
    with pytest.raises(SscfError) as e:
        ctx.step()
    assert e.value.status == -5
    assert np.array_equal(ctx.get_C(), C0)
    q1, dq1, Q1 = ctx.get_charges()
    assert np.array_equal(q1, q0) and np.array_equal(dq1, dq0) and np.array_equal(Q1, Q0)


@pytest.mark.gpu
def test_restart_refuses_bad_checkpoints_and_keeps_the_mos():
    from gpu_common import context, water
    from paper_1402_2880_gb300 import SscfError
    ctx = context(water(32), precision=1)
    ctx.set_thresholds(1e-5, 1e-4, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    C0 = ctx.get_C()
    nt, tiles, vals = ctx.get_C_tiles()
    bad = vals.copy()
    bad[5, 2, 3] = np.inf
    with pytest.raises(SscfError) as e:
        ctx.set_C_tiles(nt, tiles, bad)
    assert e.value.status == -4
    assert np.array_equal(ctx.get_C(), C0)
    unsorted = tiles.copy()
    unsorted[[0, 1]] = unsorted[[1, 0]]
    with pytest.raises(SscfError) as e:
        ctx.set_C_tiles(nt, unsorted, vals)
    assert e.value.status == -1
    assert np.array_equal(ctx.get_C(), C0)
    ctx.step()
    ctx.set_C_tiles(nt, tiles, vals)                 # restart from the checkpoint
    assert np.array_equal(ctx.get_C(), C0)
