"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.  Each rank runs an
independent replica; the whole-job value is the units of all ranks over the slowest
rank's time."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [100.0, 250.0][rank]
    local_units = [1e6, 3e6][rank]
    ups, ms = bench.aggregate(local_ms, local_units)
    out[rank] = (ups, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ups, ms = res[rank]
        assert ms == pytest.approx(250.0)
        assert ups == pytest.approx(4e6 / 0.25)


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench

    ups, ms = bench.aggregate(50.0, 1e6)
    assert ms == 50.0 and ups == pytest.approx(2e7)
