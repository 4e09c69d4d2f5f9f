"""The replica path's host logic at world size 2 on CPU (gloo): the timed
region's length is the slowest rank's, the value counts every rank's frames,
and the reference arm runs on rank 0 only (the others return without work)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, "cpu")
        value = bench.whole_job_value(64 * 3, w, ms)
        dist.barrier()
        out.put((r, w, local, ms, value, bench.run_reference(None, None) if r != 0 else "rank0"))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, ms, value, ref) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        assert ms == 15.0                                  # the slower rank's time on every rank
        assert value == pytest.approx(64 * 3 * world / 0.015)
        assert ref == ("rank0" if r == 0 else None)         # reference arm: rank 0 alone


def test_single_rank_keeps_its_time():
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.whole_job_value(100, 1, 50.0) == pytest.approx(2000.0)
