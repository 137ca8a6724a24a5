"""The N > 1 path of bench.py on the CPU: two gloo ranks, each running its own replica.

The bench runs one independent replica per GPU (the path is not sharded) and reports the
whole-job time per stage: the slowest rank's total time over all the stages the ranks ran.
This checks the max-over-ranks reduction and that quotient with two processes on the host,
as the launcher would start them (RANK / WORLD_SIZE / LOCAL_RANK from the environment).
"""
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


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.env_rank()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        t_local = [3.0, 5.0][r]  # the second replica is the slower one
        t_max = bench.max_over_ranks(t_local, w, "cpu")
        out.put((r, w, local, t_max, bench.job_seconds_per_stage(t_max, 5, w)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(out.get(timeout=10) for _ in range(2))
    for r, (rank, world, local, t_max, sps) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t_max == 5.0  # both ranks see the slowest replica's time
        assert sps == 5.0 / (5 * 2)  # ten stages ran in the job's 5 s


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_seconds_per_stage(2.5, 5, 1) == 0.5
