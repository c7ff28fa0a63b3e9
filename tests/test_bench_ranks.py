"""Host logic of the benchmark's multi-rank path (one replica per rank, max-over-ranks
timing, whole-job rate), run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 2.0 + 3.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(my_ms, world, device="cpu")
        second = bench.max_over_ranks(10.0 - rank, world, device="cpu")
        bench.barrier(world, cuda=False)
        out.put((rank, ms, second, bench.whole_job_rate(world, 1000.0, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, second, rate in got:
        assert ms == 5.0 and second == 10.0
        assert rate == pytest.approx(2 * 1000.0 / 5.0e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 500.0, 2.0) == pytest.approx(250000.0)
