"""Column partition of the circuit-unitary chain across ranks.

Column j of U = S_m ... S_1 is the circuit applied to |j> (Algorithm 1 acts on
each column alone), so the chain shards by column blocks with no exchange:
every rank generates each S_k from the circuit's step table and multiplies
its own block.  Blocks are whole tensor-core tiles (128 columns) from n = 7
on, single columns below; ranks get contiguous runs of tiles whose sizes
differ by at most one tile (a rank may get none when there are fewer tiles
than ranks).
"""
from __future__ import annotations

from typing import List, Tuple

TILE = 128


def block_unit(n: int) -> int:
    """Columns per indivisible unit of the partition."""
    return TILE if n >= 7 else 1


def column_blocks(n: int, world: int) -> List[Tuple[int, int]]:
    """(col0, ncols) of every rank, in rank order; they tile [0, 2^n)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    unit = block_unit(n)
    units = (1 << n) // unit
    out = []
    for r in range(world):
        u0 = units * r // world
        u1 = units * (r + 1) // world
        out.append((u0 * unit, (u1 - u0) * unit))
    return out


def rank_block(n: int, rank: int, world: int) -> Tuple[int, int]:
    """(col0, ncols) of this rank (ncols may be 0)."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return column_blocks(n, world)[rank]
