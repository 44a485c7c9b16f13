"""The multi-GPU bench path is replicas: each rank simulates its own seeded
batch and the ranks exchange only the timing (max over ranks).  This runs that
host logic with two gloo ranks on the CPU (no GPU, no NCCL)."""
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


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2305_14398_gb300 import workloads as W

        circs = bench.replica_circuits(W, rank, 8)
        # each rank's "elapsed seconds" differ; the job rate uses the slowest
        seconds = 0.5 + rank
        slowest = bench.max_over_ranks(seconds, dist, "cpu")
        rate = bench.whole_job_rate(len(circs), world, slowest)
        first_ops = repr(circs[3][1][:4])
        q.put((rank, slowest, rate, first_ops))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, slowest, rate, _ in res:
        assert slowest == 1.5            # max over ranks
        assert rate == 8 * 2 / 1.5       # all ranks' circuits / slowest rank's time
    # ranks draw different seeded circuits (no shared work, no data exchange)
    assert res[0][3] != res[1][3]
