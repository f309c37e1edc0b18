"""Host logic of the multi-GPU bench path, run as two gloo ranks on the CPU.

Independent clusters are sharded over ranks with no collective on the data
path; the only collectives are the two reductions of the measurement: the
whole-job atom count (sum) and the slowest rank's time (max).
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [300, 1200, 2500, 800, 640]
        mine = bench.shard(enumerate(sizes), rank, world)
        atoms = sum(3 * n for _, n in mine)
        total, t_max = bench.aggregate(atoms, 10.0 + rank, dist, "cpu")
        out[rank] = (tuple(k for k, _ in mine), total, t_max)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_clusters_and_reduce_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == (0, 2, 4) and res[1][0] == (1, 3)
    total = 3 * (300 + 1200 + 2500 + 800 + 640)
    for r in range(world):
        assert res[r][1] == pytest.approx(total)
        assert res[r][2] == pytest.approx(11.0)


def test_single_process_aggregate_is_identity():
    assert bench.aggregate(123, 4.5) == (123.0, 4.5)
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
