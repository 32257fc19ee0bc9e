"""The benchmark's multi-GPU logic on CPU: two gloo ranks shard the headline
workload (weak scaling, no data-path collective) and agree on the job's step
time as the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    pats = bench.rank_patterns(world, rank)
    t = [10.0 + rank, 5.0 - rank]  # fake per-rank step / kernel times
    m = bench.max_over_ranks(dist, "cpu", *t)
    out[rank] = (np.concatenate(pats).tolist(), len(pats), m)
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import bench
    import workloads as W

    assert res[0][1] == res[1][1] == 4096
    # rank 0 of a one-GPU run and of a two-GPU run get the headline batch
    single = np.concatenate(W.workload("batched_m64_n16")[2]).tolist()
    assert res[0][0] == single
    assert res[0][0] != res[1][0]  # disjoint draws
    assert res[0][2] == res[1][2] == [11.0, 5.0]  # max over ranks, every rank sees it
    assert bench.max_over_ranks(None, "cpu", 1.0, 2.0) == [1.0, 2.0]
