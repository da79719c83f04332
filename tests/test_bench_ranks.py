"""Host logic of the multi-GPU bench (replicas, one process per GPU), run as
world-size-2 gloo ranks on the CPU: the barrier around the timed region, the
max of the step times over the ranks, and the whole-job throughput."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier()
        # each rank's own (step ms, end-to-end ms); the job takes the slowest of each
        mine = [2.0 + rank, 5.0 - 2.0 * rank]
        got = bench.max_over_ranks(mine, "cpu")
        bench.barrier()
        out.put((rank, got, bench.job_throughput(world, got[0])))
    finally:
        dist.destroy_process_group()


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks([1.5, 2.5], "cpu") == [1.5, 2.5]
    bench.barrier()  # no process group: nothing to wait for
    assert bench.job_throughput(1, 2.0) == pytest.approx(500.0)


def test_two_gloo_ranks_take_the_slowest_step():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, thr in res:
        # step ms 2.0 and 3.0 -> 3.0; end-to-end ms 5.0 and 3.0 -> 5.0 on every rank
        assert got == [3.0, 5.0], (rank, got)
        # two replicas, one step each per 3 ms: 666.7 iterations per second for the job
        assert thr == pytest.approx(2 * 1000.0 / 3.0)
