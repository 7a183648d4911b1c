"""The benchmark's N > 1 path (replicas only: one independent copy of the workload per rank,
no collective on the data path) on CPU with world size 2 over gloo: the job's step time is the
largest over the ranks and the job's rate counts every rank's bytes; the reference arm runs on
rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [3.0, 5.5][rank]
        job_ms = bench._max_over_ranks(local_ms, world, "cpu")
        rate = bench._job_rate(world, 6.0e9, job_ms)
        q.put((rank, job_ms, rate))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_all_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [5.5, 5.5]
    assert out[0][2] == pytest.approx(2 * 6.0e9 / 5.5e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(4.25, 1) == 4.25
    assert bench._job_rate(1, 1.0e9, 1.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, rank=1, world=2) is None  # returns before any work
