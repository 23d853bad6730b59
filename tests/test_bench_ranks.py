"""Host logic of multi-GPU runs, on CPU with world_size 2 (gloo): every rank
gets independent chains and the job's throughput is the sum of the ranks'
units over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms_local = 10.0 + 5.0 * rank            # rank 1 is slower
    units = 1000 * (rank + 1)
    ms, value = bench.aggregate(ms_local, units, ws)
    out[rank] = (ms, value, bench.rank_seed(7, rank))
    dist.destroy_process_group()


def test_two_ranks_aggregate_and_independent_seeds():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    (ms0, v0, s0), (ms1, v1, s1) = out[0], out[1]
    assert ms0 == ms1 == 15.0
    assert abs(v0 - 3000 / 0.015) < 1e-6 and v0 == v1
    assert s0 != s1


def test_single_rank_is_local():
    import bench
    ms, v = bench.aggregate(4.0, 400, 1)
    assert ms == 4.0 and v == 100000.0
