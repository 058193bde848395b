"""The multi-GPU path is replicas only (columns and frames are independent, no
exchange step).  What the ranks share is the timing: the job's time is the
slowest rank's and its throughput counts every rank's frames.  These tests run
that logic with world_size 2 on the CPU over gloo, as separate processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_info()
        slowest = bench.max_over_ranks(times[rank], w, torch.device("cpu"))
        rate = bench.job_rate(100, w, slowest)
        dist.barrier()
        out_q.put((r, local, w, slowest, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.5, 2.0), (3.0, 1.0)])
def test_two_ranks_take_the_slowest_time_and_count_all_frames(times):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, (r, local, w, slowest, rate) in enumerate(got):
        assert (r, local, w) == (rank, rank, 2)
        assert slowest == max(times)
        assert rate == pytest.approx(200 / max(times))


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1.25, 1, None) == 1.25
    assert bench.job_rate(300, 1, 0.5) == 600
