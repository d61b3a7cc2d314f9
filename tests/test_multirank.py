"""The N > 1 path of bench.py on the CPU: two gloo ranks agree on the
slowest rank's time and the whole-job throughput counts the units of all
ranks (weak scaling).  No GPU: the data path has no collective, only this
timing reduction."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [40.0, 55.0][rank]            # per-rank elapsed milliseconds
        worst = bench.max_over_ranks(ms)
        out.put((rank, worst, bench.job_throughput(2000, 10, world, worst)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, thr in res:
        assert worst == 55.0
        assert thr == pytest.approx(2000 * 10 * 2 / 0.055)


def test_single_process_is_the_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(100, 4, 1, 200.0) == pytest.approx(2000.0)
