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


@pytest.mark.parametrize("n,prec", [(32, 0), (32, 1)])
def test_graph_resident_run_equals_host_loop(n, prec):
    """With graphs enabled, each SCC stage of sscf_run is one graph launch whose
    while node repeats the iteration until the device-side test says stop: the
    same iterations, energies, charges and MOs as the host-driven loop."""
    import torch
    s = water(n)
    stream = torch.cuda.Stream()
    outs = []
    for graph in (False, True):
        c = context(s, precision=prec, stream=stream.cuda_stream)
        if graph:
            c.enable_graph(True)
        r = c.run()
        q, _, _ = c.get_charges()
        outs.append((r, q, c.get_C()))
    (ra, qa, Ca), (rb, qb, Cb) = outs
    assert ra["converged"] and rb["converged"]
    assert ra["iteration"] == rb["iteration"]
    assert ra["energy"] == rb["energy"]
    assert np.array_equal(qa, qb) and np.array_equal(Ca, Cb)


def test_graph_resident_batch_run():
    import torch

    from gpu_common import library
    library()
    from synth import concat_clusters, lattice_water
    s = concat_clusters([lattice_water(8, seed=4), lattice_water(16, seed=5), lattice_water(32, seed=0)])
    stream = torch.cuda.Stream()
    res = []
    for graph in (False, True):
        c = context(s, stream=stream.cuda_stream)
        if graph:
            c.enable_graph(True)
        r = c.run()
        e, d = c.cluster_results()
        res.append((r["converged"], r["iteration"], e))
    assert res[0][0] and res[1][0]
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2])
