"""The N-rank timing of bench.py (replicas: every rank runs the same workload) with world_size-2
gloo process groups on the CPU: every rank reports the slowest rank's time, and the whole-job value
counts the units of all ranks over that time."""
import importlib.util
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, times, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = b.max_over_ranks(times[rank], world, "cpu")
    value = b.job_value(world, 1000.0, ms)
    dist.destroy_process_group()
    q.put((rank, ms, value))


@pytest.mark.parametrize("times", [[12.5, 20.0], [30.0, 7.25]])
def test_ranks_report_the_slowest_time(times):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    for _, ms, value in results:
        assert ms == slowest
        assert value == pytest.approx(world * 1000.0 / (slowest / 1e3), rel=1e-15)


def test_single_rank_is_its_own_time():
    b = _bench()
    assert b.max_over_ranks(3.5, 1) == 3.5
    assert b.job_value(1, 500.0, 250.0) == pytest.approx(2000.0)
