"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2): the path
shards into independent replicas, one per rank, so the only collectives are the
barrier and the maximum of the per-rank times, and the job's throughput is the
sum over replicas in the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]  # the second rank is the slow one
        dist.barrier()
        worst = bench.max_over_ranks(ms, world)
        out.put((rank, worst, bench.job_mlups(2048 * 1024, 1000, worst, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, mlups in res:
        assert worst == 17.25
        assert mlups == pytest.approx(2 * 2048 * 1024 * 1000 / 17.25e-3 / 1e6)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_mlups(100, 10, 1.0, 1) == pytest.approx(1.0)
