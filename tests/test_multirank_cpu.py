"""Host logic of bench.py's multi-GPU mode on CPU: two gloo ranks run
independent replicas (no data-path collective); the whole-job value is the
units both ranks processed over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pushes = [1000, 3000][rank]
    ms = [10.0, 40.0][rank]
    value, tmax = bench.aggregate(dist, pushes, ms)
    out[rank] = (value, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_is_total_over_slowest():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, tmax = res[r]
        assert tmax == pytest.approx(40.0)
        assert value == pytest.approx(4000 / 40e-3)


def test_single_process_aggregate():
    import bench
    v, t = bench.aggregate(None, 500, 5.0)
    assert v == pytest.approx(1e5) and t == 5.0
