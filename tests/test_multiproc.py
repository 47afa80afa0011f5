"""Replica path of bench.py (one independent instance per rank) on CPU ranks
with the gloo backend, world size 2: the whole-job time is the slowest
rank's, the beam states are summed, and ranks solve distinct instances."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, cand = bench.aggregate_over_ranks(100.0 * (rank + 1), 1.0e6 * (rank + 1))
    import instances
    seed = bench.rank_instance_seed(rank)
    inst = instances.chimera(2, seed)
    out[rank] = (ms, cand, seed, float(inst.J.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 200.0          # max over ranks
    assert res[0][1] == res[1][1] == 3.0e6          # sum over ranks
    assert res[0][2] != res[1][2]                   # independent instances
    assert res[0][3] != res[1][3]
