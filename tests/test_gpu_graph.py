"""CUDA-graph steps (sscf_enable_graph) replay exactly the eager step."""
import numpy as np
import pytest

from gpu_common import context, water

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,prec", [(32, 0), (216, 1)])
def test_graph_steps_equal_eager_steps(n, prec):
    import torch
    s = water(n)
    stream = torch.cuda.Stream()
    ctxs = []
    for graph in (False, True):
        c = context(s, precision=prec, stream=stream.cuda_stream)
        c.set_thresholds(1e-5, 1e-4, 1e-8)
        c.guess()
        c.orthonormalise(0)
        c.reset_charges()
        if graph:
            c.enable_graph(True)
        ctxs.append(c)
    for k in range(3):
        a, b = ctxs[0].step(), ctxs[1].step()
        assert a["energy"] == b["energy"] and a["n_rot"] == b["n_rot"] and a["n_combo"] == b["n_combo"]
        assert b["launches"] == a["launches"]
    qa, _, _ = ctxs[0].get_charges()
    qb, _, _ = ctxs[1].get_charges()
    assert np.array_equal(qa, qb)
    assert np.array_equal(ctxs[0].get_C(), ctxs[1].get_C())


def test_graph_needs_a_stream():
    from paper_1402_2880_gb300 import SscfError
    c = context(water(8))
    with pytest.raises(SscfError):
        c.enable_graph(True)
