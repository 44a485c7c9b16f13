"""The column-sharded chain's partition (paper_2305_14398_gb300.shard) on two
gloo ranks on the CPU: each rank takes its block of columns of the circuit
unitary, computes it alone (here with the FP64 oracle's column route, eq. 12
applied to |j>, standing in for the GPU call), and the blocks gathered on
rank 0 tile the columns and put side by side equal the whole unitary
(Algorithm 1).  No exchange happens before the gather."""
import os
import socket

import numpy as np
import pytest

from paper_2305_14398_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import fsv_route
        from paper_2305_14398_gb300 import workloads as W

        ops = W.random_layered(n, 3, (93, n))
        col0, ncols = shard.rank_block(n, rank, world)
        blk = fsv_route.unitary_columns(n, ops, list(range(col0, col0 + ncols)))
        t = torch.from_numpy(np.ascontiguousarray(blk.T))  # rows = this rank's columns
        sizes = [None] * world
        dist.all_gather_object(sizes, (col0, ncols))
        parts = [torch.empty((s[1], 1 << n), dtype=t.dtype) for s in sizes]
        dist.all_gather(parts, t)
        if rank == 0:
            U = torch.cat(parts).numpy().T
            q.put((sizes, float(np.max(np.abs(U - fsv_route.unitary_columns(n, ops, list(range(1 << n))))))))
    finally:
        dist.destroy_process_group()


def test_column_blocks_tile_the_columns():
    for n in range(1, 15):
        for world in (1, 2, 3, 4, 8, 200):
            blocks = shard.column_blocks(n, world)
            assert len(blocks) == world
            nxt = 0
            for col0, ncols in blocks:
                assert col0 == nxt and ncols >= 0
                assert col0 % shard.block_unit(n) == 0 and ncols % shard.block_unit(n) == 0
                nxt = col0 + ncols
            assert nxt == 1 << n
            sizes = [b[1] for b in blocks]
            assert max(sizes) - min(sizes) <= shard.block_unit(n)


@pytest.mark.parametrize("n", [8, 5])
def test_two_gloo_ranks_blocks_gather_to_the_unitary(n):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sizes, err = q.get(timeout=10)
    assert sizes == shard.column_blocks(n, world)
    assert err == 0.0
