"""The benchmark's multi-rank path on CPU: two gloo ranks (replicas of the workload, no
exchange on the data path) reduce their timings to the slowest rank's, and the whole-job rate
counts every rank's solves."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        import bench
        # rank r "took" 10 + r ms per step and 1 + 2r s of wall time
        dev_ms, wall = bench.max_over_ranks([10.0 + rank, 1.0 + 2.0 * rank], world, "cpu")
        rate = bench.whole_job_rate(world, 5, dev_ms / 1000.0)
        dist.barrier()
        q.put((rank, dev_ms, wall, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dev_ms, wall, rate in out:
        assert dev_ms == 11.0 and wall == 3.0            # every rank sees the slowest rank's times
        assert rate == pytest.approx(2 * 5 / 0.011)      # all ranks' solves over the slowest time


def test_single_rank_is_the_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 10, 0.5) == 20.0
