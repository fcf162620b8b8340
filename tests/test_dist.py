"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each an independent
replica (no data-path collective); timing is the maximum over ranks and the reported
throughput counts the units of every rank."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    assert bench._dist() == (world, rank)
    ms_local = 10.0 + 5.0 * rank          # the second rank is slower
    ms = bench.max_over_ranks(ms_local)
    rate = bench.whole_job_rate(1000 * 20, world, ms)
    dist.barrier()
    out[rank] = (ms, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 * 20 / 0.015)


def test_single_process_is_its_own_maximum():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(100, 1, 1000.0) == 100.0
