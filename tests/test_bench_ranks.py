"""The replicas-only multi-GPU path of bench.py on CPU: two gloo ranks report
the whole-job rate over the slowest rank (no data-path collective)."""
import os
import socket
import sys

import pytest

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
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    cells = [1000, 3000][rank]
    ms = [5.0, 8.0][rank]
    rate, mx, total = bench.whole_job_rate(cells, 10, ms, dist, "cpu")
    out[rank] = (rate, mx, total)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        rate, mx, total = res[rank]
        assert mx == 8.0 and total == 4000
        assert rate == pytest.approx(4000 * 10 / 8e-3 / 1e6)


def test_whole_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    rate, mx, total = bench.whole_job_rate(2000, 5, 4.0)
    assert (mx, total) == (4.0, 2000) and rate == pytest.approx(2000 * 5 / 4e-3 / 1e6)
