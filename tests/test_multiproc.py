"""The multi-GPU launch is replicas only (every rank tracks its own synthetic frame, with
no data-path collective): the host logic that joins the ranks -- max-over-ranks timing and
the whole-job rate -- on two gloo ranks on the CPU, and the reference arm's rank split."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # the second replica is slower
    ms_max = bench.max_over_ranks(ms, world, "cpu")
    rate = bench.whole_job_rate(307200, 100, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, rate))


def test_replicas_join_on_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms_max, rate in got:
        assert ms_max == 15.0
        # both replicas' units over the slowest replica's time
        assert rate == pytest.approx(2 * 100 * 307200 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 4, 1, 2.0) == pytest.approx(20000.0)
