"""Windowed closures (closure_mode = k >= 1) against the per-sweep closure.

Both place tiles before the 2x2 updates of a sweep and neither changes a
value, so C, the pair lists and every energy must agree bit for bit. A
window of k colours gives a row only the tiles its units are connected to
through those colours' active blocks, counting only units it holds nonzero
values in, so rows hold their real fill plus one window's insertions: with a
row capacity far below the cluster's tile count it still runs the passes that
the per-sweep closure (which gives a row every tile its units are connected
to) refuses with SSCF_ERR_CAPACITY (window of 1 colour; with every block
active, as in the first orthonormalisation from the guess, a window of many
colours links units across most of the cluster and needs room for that
transient fill). Bit-identity is checked for windows of 1 and 8 colours.
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


@pytest.mark.parametrize("n,precision,window", [(100, 0, 1), (216, 1, 1), (216, 1, 8)])
def test_windowed_closure_gives_the_same_mos(n, precision, window):
    _, a = _trajectory(n, precision, 0)
    _, b = _trajectory(n, precision, window)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    assert a[3:-1] == b[3:-1]
    assert np.array_equal(a[-1], b[-1])


def test_per_colour_closure_fits_where_the_sweep_closure_overflows():
    """4096 molecules after the guess and the loose full orthonormalisation
    (eps 1e-3, the bench's input state), then one SCC iteration: the MOs are
    local, so rows hold a few hundred of the 1536 tiles. With 640 tiles per row
    the per-sweep closure overflows on the first pass (it gives a row every
    tile of the cluster); the per-colour closure runs, and its checkpoint of C
    equals the dense-row reference tile for tile."""
    from paper_1402_2880_gb300 import SscfError
    s = water(4096)

    def prep(closure_mode, cap_tiles):
        ctx = context(s, precision=1, closure_mode=closure_mode, cap_tiles=cap_tiles)
        ctx.set_thresholds(1e-3, 1e-2, 1e-8)
        ctx.guess()
        ctx.orthonormalise(0)
        first = ctx.get_C_tiles()
        ctx.set_thresholds(1e-5, 1e-4, 1e-6)
        ctx.reset_charges()
        info = ctx.step()
        return first, ctx.get_C_tiles(), info

    ref_first, ref_after, ref_info = prep(0, 0)
    cap = 640
    print(f"rows hold at most {ref_first[0].max()} tiles after the orthonormalisation and "
          f"{ref_after[0].max()} after one iteration; capacity {cap}")
    assert ref_after[0].max() < cap
    with pytest.raises(SscfError) as e:
        prep(0, cap)
    assert e.value.status == -5
    got_first, got_after, got_info = prep(1, cap)
    for a, b in ((got_first, ref_first), (got_after, ref_after)):
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert got_info["energy"] == ref_info["energy"]
