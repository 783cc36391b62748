"""Multi-rank logic of bench.py on CPU: two gloo ranks.

Weak scaling shards targets across ranks with no collective in the data path: every
rank builds the same surface with its own seeded target set, and the only
collectives are the max (step time) and sum (entries) reductions of the timing.
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


def _rank_main(rank: int, world: int, port: int, outdir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    mx = bench.reduce_max(1.5 + rank, w)
    sm = bench.reduce_sum(1.5 + rank, w)
    d, tg = bench.workload(r, ntarg=64)
    # the reference arm: only rank 0 works and prints; the others return at once
    class A:
        steps, warmup, cpu_targets = 1, 0, 4
    ref_ran = False
    if rank != 0:
        bench.bench_reference(A())
        ref_ran = True
    dist.barrier()
    dist.destroy_process_group()
    np.savez(os.path.join(outdir, f"r{rank}.npz"), xyz=d.xyz, txyz=tg.xyz, tself=tg.self_node,
             meta=json.dumps(dict(rank=r, world=w, local=lr, mx=mx, sm=sm, ref_ran=ref_ran)))


def test_two_rank_weak_scaling_logic(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    meta = [json.loads(str(x["meta"])) for x in res]
    for r, m in enumerate(meta):
        assert (m["rank"], m["world"], m["local"]) == (r, world, r)
        assert m["mx"] == pytest.approx(2.5)       # max over ranks of 1.5 + rank
        assert m["sm"] == pytest.approx(4.0)       # sum over ranks
    assert meta[1]["ref_ran"]
    # same surface on every rank, distinct seeded target sets (weak scaling shards)
    np.testing.assert_array_equal(res[0]["xyz"], res[1]["xyz"])
    assert res[0]["txyz"].shape == res[1]["txyz"].shape == (64, 3)
    assert not np.allclose(res[0]["txyz"], res[1]["txyz"])
    assert np.all(res[0]["tself"] == -1) and np.all(res[1]["tself"] == -1)


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25, 1) == 3.25
    assert bench.reduce_sum(3.25, 1) == 3.25
