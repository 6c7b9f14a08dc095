"""The multi-rank bench path: replicas combined over a gloo process group on CPU.

bench.py runs one independent replica per rank (the path does not shard);
the whole-job figure is all ranks' work over the slowest rank's time.  Two
ranks with different times must agree on that figure.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
        local_flop = 1_000_000 * (rank + 1)
        out[rank] = bench.combine_replicas(local_ms, local_flop, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_slowest_time_and_total_work():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    slowest_ms = 20.0
    total_flop = 1_000_000 + 2_000_000
    for r in range(world):
        ms, gflops = res[r]
        assert ms == pytest.approx(slowest_ms)
        assert gflops == pytest.approx(2.0 * total_flop / (slowest_ms / 1e3) / 1e9)


def test_single_process_is_its_own_figure():
    sys.path.insert(0, ROOT)
    import bench
    ms, gflops = bench.combine_replicas(4.0, 1_000_000, "cpu")
    assert ms == 4.0 and gflops == pytest.approx(2.0 * 1e6 / 4e-3 / 1e9)
