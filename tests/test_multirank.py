"""Multi-rank logic on CPU: two gloo ranks.

Row-block sharding of one problem: the targets split into contiguous blocks, one per
rank; each rank builds the CSR rows of its block against the whole geometry, with no
collective in the data path (the bench's only collectives are the max of the step time
and the sum of the entries).  Here the oracle stands in for the per-rank GPU build (test
only): the blocks must cover every row exactly once, and the concatenated blocks, row
pointers rebased, must equal the single-rank CSR bit for bit.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_2411_08342_gb300 import workloads as W
    d = W.discretize(W.star_surface(1), 4)
    on = W.on_surface_targets(d)
    return d, W.concat_targets(on, W.off_surface_targets(d, 301, seed=5))


def _rank_main(rank: int, world: int, port: int, outdir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), OMP_NUM_THREADS="2")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from oracle import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    mx = bench.reduce_max(1.5 + rank, w)
    sm = bench.reduce_sum(1.5 + rank, w)
    d, tg = _problem()
    blk, (lo, hi) = bench.rank_targets(tg, r, w)
    # the oracle as the CPU stand-in of this rank's block build
    rp, col, vals, _ = oracle.OracleSurface(d).csr_rows(blk)
    gathered = [None] * w
    dist.all_gather_object(gathered, (lo, hi, rp, col, vals))
    # the reference arm: only rank 0 works and prints; the others return at once
    class A:
        steps, warmup, cpu_targets, ref_targets = 1, 0, 4, 4
    ref_ran = False
    if rank != 0:
        bench.bench_reference(A())
        ref_ran = True
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        np.save(os.path.join(outdir, "blocks.npy"), np.array(gathered, dtype=object), allow_pickle=True)
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump(dict(rank=r, world=w, local=lr, mx=mx, sm=sm, ref_ran=ref_ran, lo=lo, hi=hi), f)


def test_two_rank_row_blocks(tmp_path, oracle_lib):
    from paper_2411_08342_gb300.shard import concat_row_blocks
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    meta = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r, m in enumerate(meta):
        assert (m["rank"], m["world"], m["local"]) == (r, world, r)
        assert m["mx"] == pytest.approx(2.5)       # max over ranks of 1.5 + rank
        assert m["sm"] == pytest.approx(4.0)       # sum over ranks
    assert meta[1]["ref_ran"]
    d, tg = _problem()
    # the blocks cover every row once, in order
    assert meta[0]["lo"] == 0 and meta[0]["hi"] == meta[1]["lo"] and meta[1]["hi"] == tg.n
    blocks = np.load(tmp_path / "blocks.npy", allow_pickle=True)
    rp, col, vals = concat_row_blocks([(b[2], b[3], b[4]) for b in blocks])
    srp, scol, svals, _ = oracle_lib.OracleSurface(d).csr_rows(tg)
    assert np.array_equal(rp, srp) and np.array_equal(col, scol)
    for k in svals:
        assert np.array_equal(vals[k], svals[k]), k


@pytest.mark.parametrize("n,world", [(0, 3), (1, 4), (10, 3), (1_720_320, 8), (937_280, 7)])
def test_row_block_partition(n, world):
    from paper_2411_08342_gb300.shard import row_block
    bounds = [row_block(n, r, world) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == n
    for (a, b), (c, e) in zip(bounds, bounds[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in bounds]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25, 1) == 3.25
    assert bench.reduce_sum(3.25, 1) == 3.25
