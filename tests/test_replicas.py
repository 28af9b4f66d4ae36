"""The replica path of bench.py on two gloo ranks (CPU): the job's time is the
slowest rank's and the value counts every rank's iterations."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 * (rank + 1)           # rank 1 is the slower replica
    t = bench.max_over_ranks(ms, world, torch.device("cpu"))
    out[rank] = (t, bench.job_value(500, 3, world, t))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        t, v = res[r]
        assert t == 200.0
        assert v == pytest.approx(500 * 3 * 2 / 0.2)
