"""The allocation-free pair selection agrees with the selection inside sscf_rotate_sweep.

For callers that cannot allocate device memory, sscf_select_pairs_noalloc
applies the rotation-pair rule of a sweep to arrays they own, with its
working memory in a file-scope device array. This file runs last: it checks
two calls in a row against the pairs the regular entry point chose from the
same F values and against the oracle's selection rule on those values, and
that oversized inputs are refused.
"""
import numpy as np
import pytest

from gpu_common import P, context, oracle_scf, water
from oracle import sparse

pytestmark = pytest.mark.gpu


def _noalloc_keep(F, eps, k_max):
    import torch

    from paper_1402_2880_gb300 import _lib
    f = torch.from_numpy(np.ascontiguousarray(F, dtype=np.float64).ravel()).cuda()
    keep = torch.full((f.numel(),), 7, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    n_keep = _lib.select_pairs_noalloc(f.data_ptr(), f.numel(), eps, k_max, keep.data_ptr(), stream)
    torch.cuda.synchronize()
    return keep.cpu().numpy().reshape(F.shape).astype(bool), n_keep


def test_noalloc_selection_matches_rotate_sweep_twice():
    n = 216
    eps = 1e-6
    ctx = context(water(n))
    ctx.set_thresholds(eps, 10 * eps, 1e-8)
    ctx.guess()
    ctx.orthonormalise(0)
    rng = np.random.default_rng(11)
    ctx.set_charges(Q_in=rng.normal(0.0, 0.2, water(n).n_atoms))
    k_max = int(P["rot_cap_factor"] * ctx.n_occ)
    capped = []
    for call in range(2):
        ctx.build_fock()
        n_rot, _ = ctx.rotate_sweep()              # the regular entry point
        F, _ = ctx.get_F()
        _, _, i, j = ctx.pairs()
        want = np.zeros(F.shape, dtype=bool)
        want[i, j - ctx.n_occ] = True
        got, n_keep = _noalloc_keep(F, eps, k_max)
        assert n_keep == n_rot == int(want.sum())
        assert np.array_equal(got, want), f"call {call}"
        st = oracle_scf(n).st
        mask = st.group_nb[st.mo_group[:st.n_occ][:, None], st.mo_group[st.n_occ:][None, :]]
        assert np.array_equal(got, sparse.select_pairs(F, mask, eps, k_max)), f"call {call}"
        capped.append(int(((np.abs(F) >= eps) & (F != 0)).sum()) > k_max)
    assert any(capped), "at least one call must exercise the top-k cap"


def test_noalloc_rejects_oversized_input():
    import torch

    from paper_1402_2880_gb300 import SscfError, _lib
    f = torch.zeros(4, dtype=torch.float64, device="cuda")
    keep = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(SscfError) as e:
        _lib.select_pairs_noalloc(f.data_ptr(), (1 << 21) + 1, 1e-6, 10, keep.data_ptr())
    assert e.value.status == -1
    assert _lib.select_pairs_noalloc(f.data_ptr(), 4, 1e-6, 10, keep.data_ptr()) == 0
