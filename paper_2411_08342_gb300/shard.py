"""Row-block sharding of one correction build over several processes (one GPU each).

The near pairs of different targets are independent (Sec. 4: every (target, patch) pair
is computed on its own), so the rows of one problem split into contiguous blocks, one
per rank, with no exchange in the build: every rank holds the whole geometry and builds
the CSR rows of its block of targets.  Applying the corrections needs the whole density
on every rank (columns are global node ids); it is an input, so each rank holds a copy.

Host logic only: the block bounds, and the reassembly of per-rank CSR blocks into the
CSR of the whole problem (row pointers rebased, columns and values concatenated).
"""
from __future__ import annotations

import numpy as np


def row_block(ntarg: int, rank: int, world: int) -> tuple[int, int]:
    """Targets [lo, hi) of rank `rank` out of `world`: contiguous, sizes differing by at
    most one, the larger blocks first; every target in exactly one block."""
    if world < 1 or not 0 <= rank < world or ntarg < 0:
        raise ValueError("bad rank/world/ntarg")
    q, r = divmod(ntarg, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def concat_row_blocks(blocks):
    """CSR of the whole problem from the per-rank blocks in rank order, each block a
    (rowptr, col, {kernel: val}) with rowptr starting at 0."""
    rps, cols, vals = [], [], {}
    off = 0
    for i, (rp, col, v) in enumerate(blocks):
        rp = np.asarray(rp, np.int64)
        if rp[0] != 0:
            raise ValueError("block row pointers must start at 0")
        rps.append(rp[(1 if i else 0):] + off)
        off += int(rp[-1])
        cols.append(np.asarray(col)[: int(rp[-1])])
        for k, a in v.items():
            vals.setdefault(k, []).append(np.asarray(a)[: int(rp[-1])])
    rowptr = np.concatenate(rps) if rps else np.zeros(1, np.int64)
    return rowptr, np.concatenate(cols) if cols else np.zeros(0, np.int32), \
        {k: np.concatenate(a) for k, a in vals.items()}
