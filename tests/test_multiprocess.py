"""The multi-replica timing path of bench.py on CPU with the gloo backend,
world size 2 (the method shards into independent replicas; the only
cross-rank step is the max of the timed region)."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 100 (r + 1) ms for 1e9 updates
    ms, value, w = bench.aggregate(100.0 * (rank + 1), 1e9, dist, "cpu")
    out[rank] = (ms, value, w)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_world2_gloo():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, value, w = res[r]
        assert w == 2
        assert ms == pytest.approx(200.0)              # the slowest rank
        assert value == pytest.approx(2 * 1e9 / 0.2)   # whole-job updates / job time


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(50.0, 1e9) == (50.0, 1e9 / 0.05, 1)
