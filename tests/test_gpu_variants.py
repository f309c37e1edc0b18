"""The specialised sweep kernels give the same results as the generic one.

The rotation sweep and the occupied orthonormalisation pass of the mixed path
run blocks between two full groups (32 occupied MOs per side) through a
register-resident kernel. It applies the same FP32 updates in the same order
with the same truncation, so C must agree bit for bit with the generic kernel
(`apply_variant = 1`). `apply_variant = 2` runs the specialised kernel with one
CTA per block, so that every CTA collects row pairs with work over all of the
block's row chunks and runs them in batches of a CTA's worth (at these sizes
the default launch gives each CTA one chunk). Sizes: 216 molecules (27 full
groups: every block takes the specialised kernel) and 100 molecules (ragged
groups: both kernels run in the same colour).
"""
import numpy as np
import pytest

from gpu_common import context, water

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [100, 216])
def test_full_block_kernel_matches_generic(n):
    s = water(n)
    runs = []
    for variant in (0, 1, 2):
        ctx = context(s, precision=1, apply_variant=variant)
        ctx.set_thresholds(1e-3, 1e-2, 1e-8)
        ctx.guess()
        ctx.orthonormalise(0, max_pass=50)
        ctx.set_thresholds(1e-5, 1e-4, 1e-6)
        ctx.reset_charges()
        infos = [ctx.step() for _ in range(3)]
        passes, eta = ctx.orthonormalise(1, max_pass=2)
        runs.append((ctx.get_C(), infos, eta, ctx.get_charges()[0]))
    C0, i0, e0, q0 = runs[0]
    assert i0[-1]["n_combo"] > 0
    for C1, i1, e1, q1 in runs[1:]:
        assert np.array_equal(C0, C1)
        assert np.array_equal(q0, q1)
        assert e0 == e1
        for a, b in zip(i0, i1):
            for k in ("energy", "dq_max", "n_rot", "n_combo", "nnz_c", "upd_combo"):
                assert a[k] == b[k], k


def test_autotune_keeps_results():
    """sscf_autotune only chooses a launch shape and a register budget: the steps after it equal
    the steps of an untuned context bit for bit."""
    s = water(216)
    runs = []
    for tune in (False, True):
        ctx = context(s, precision=1)
        ctx.set_thresholds(1e-3, 1e-2, 1e-8)
        ctx.guess()
        ctx.orthonormalise(0, max_pass=50)
        ctx.set_thresholds(1e-5, 1e-4, 1e-6)
        ctx.reset_charges()
        ctx.step()
        if tune:
            assert ctx.autotune() % 16 in (1, 2, 4, 8)
        infos = [ctx.step() for _ in range(2)]
        runs.append((ctx.get_C(), infos))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert [i["energy"] for i in runs[0][1]] == [i["energy"] for i in runs[1][1]]
