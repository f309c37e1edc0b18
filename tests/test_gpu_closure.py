"""The per-colour closure (closure_mode = 1) against the per-sweep closure.

Both place tiles before the 2x2 updates of a sweep and neither changes a
value, so C, the pair lists and every energy must agree bit for bit. The
per-colour closure gives a row only the partner units of one colour's active
blocks for the units it holds nonzero values in, so rows hold their real fill
plus one colour's insertions: with a row capacity far below the cluster's
tile count it still runs the passes that the per-sweep closure (which gives a
row every tile its units are connected to) refuses with SSCF_ERR_CAPACITY.
"""
import numpy as np
import pytest

from gpu_common import context, water

pytestmark = pytest.mark.gpu


def _trajectory(n, precision, closure_mode, cap_tiles=0):
    ctx = context(water(n), precision=precision, closure_mode=closure_mode, cap_tiles=cap_tiles)
    ctx.set_thresholds(1e-3, 1e-2, 1e-8)
    ctx.guess()
    passes = ctx.orthonormalise(0)
    out = [passes, ctx.get_C()]
    ctx.set_thresholds(1e-5, 1e-4, 1e-8)
    out.append(ctx.reset_charges())
    for _ in range(3):
        info = ctx.step()
        out.append((info["energy"], info["n_rot"], info["n_combo"], info["nnz_c"]))
    out.append(ctx.get_C())
    return ctx, out


@pytest.mark.parametrize("n,precision", [(100, 0), (216, 1)])
def test_per_colour_closure_gives_the_same_mos(n, precision):
    _, a = _trajectory(n, precision, 0)
    _, b = _trajectory(n, precision, 1)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    assert a[3:-1] == b[3:-1]
    assert np.array_equal(a[-1], b[-1])


def test_per_colour_closure_fits_where_the_sweep_closure_overflows():
    from paper_1402_2880_gb300 import SscfError
    n = 512
    ref_ctx, ref = _trajectory(n, 1, 0)                       # dense rows: reference
    nt, _, _ = ref_ctx.get_C_tiles()
    n_tiles = ref_ctx.n_tiles
    cap = int(0.75 * n_tiles)
    print(f"{n_tiles} tiles, rows hold at most {nt.max()} after three iterations; capacity {cap}")
    assert nt.max() < cap                                      # the real fill fits
    with pytest.raises(SscfError) as e:
        _trajectory(n, 1, 0, cap_tiles=cap)
    assert e.value.status == -5                                # the sweep closure needs whole rows
    _, got = _trajectory(n, 1, 1, cap_tiles=cap)
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[-1], ref[-1])
    assert got[3:-1] == ref[3:-1]
