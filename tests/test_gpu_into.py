"""Builds into caller-owned buffers (rrq_build_corrections_into): page-locked host memory
written directly by the per-pair kernels, or device memory; the values must equal those
of rrq_build_corrections bit for bit.  Buffers the device cannot address (plain pageable
host memory) and too small a capacity are refused before any per-pair kernel runs."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import KINDS, gpu_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2411_08342_gb300 import rrq
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    c = rrq.Context(0)
    yield c
    c.close()


def _host(d, tg):
    return {k: np.ascontiguousarray(v) for k, v in dict(order=d.order, node_off=d.node_off, xyz=d.xyz, nrm=d.nrm,
                                                         wts=d.wts, txyz=tg.xyz, tnrm=tg.nrm,
                                                         tself=tg.self_node).items()}


@pytest.mark.parametrize("mixed", [False, True])
def test_into_pinned_host_and_device(ctx, mixed):
    import torch
    from paper_2411_08342_gb300 import rrq
    d, tg = W.star1280(6, 4000, seed=77)
    ref = gpu_build(ctx, d, tg, mixed=mixed)
    nnz = len(ref[1])
    # host inputs, pinned host outputs
    h = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in _host(d, tg).items()}
    hs = ctx.surface(h["order"], h["node_off"], h["xyz"], h["nrm"], h["wts"], d.ref_uv)
    ht = ctx.targets(h["txyz"], h["tnrm"], h["tself"])
    rp = torch.empty(tg.n + 1, dtype=torch.int64).pin_memory().numpy()
    col = torch.empty(nnz, dtype=torch.int32).pin_memory().numpy()
    vals = {k: torch.empty(nnz, dtype=torch.float64).pin_memory().numpy() for k in KINDS}
    n, npairs = ctx.build_corrections_into(hs, ht, rp, col, vals, inputs_on_host=True, mixed=mixed)
    assert n == nnz and npairs == ref[3]["npairs"]
    assert np.array_equal(rp, ref[0]) and np.array_equal(col, ref[1])
    for k in KINDS:
        assert np.array_equal(vals[k], ref[2][k]), k
    # device inputs, device outputs, one kernel
    a = rrq.device_inputs(d, tg)
    ds = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    dt = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    drp = torch.empty(tg.n + 1, dtype=torch.int64, device="cuda")
    dcol = torch.empty(nnz, dtype=torch.int32, device="cuda")
    dval = {"DP": torch.empty(nnz, dtype=torch.float64, device="cuda")}
    ctx.build_corrections_into(ds, dt, drp, dcol, dval, kernels=("DP",), mixed=mixed)
    assert np.array_equal(drp.cpu().numpy(), ref[0]) and np.array_equal(dcol.cpu().numpy(), ref[1])
    assert np.array_equal(dval["DP"].cpu().numpy(), ref[2]["DP"])


def test_into_refusals(ctx):
    import torch
    from paper_2411_08342_gb300 import rrq
    d, tg = W.sphere80(4)
    h = _host(d, tg)
    hs = ctx.surface(h["order"], h["node_off"], h["xyz"], h["nrm"], h["wts"], d.ref_uv)
    ht = ctx.targets(h["txyz"], h["tnrm"], h["tself"])
    nnz = len(gpu_build(ctx, d, tg)[1])
    # plain pageable host buffers: not addressable by the kernels
    rp, col = np.empty(tg.n + 1, np.int64), np.empty(nnz, np.int32)
    vals = {k: np.empty(nnz) for k in KINDS}
    with pytest.raises(rrq.RRQError, match="invalid argument"):
        ctx.build_corrections_into(hs, ht, rp, col, vals, inputs_on_host=True)
    # too small a capacity: refused, with the entry count reported
    prp = torch.empty(tg.n + 1, dtype=torch.int64).pin_memory().numpy()
    pcol = torch.empty(nnz, dtype=torch.int32).pin_memory().numpy()
    pvals = {k: torch.empty(nnz, dtype=torch.float64).pin_memory().numpy() for k in KINDS}
    with pytest.raises(rrq.RRQError, match="invalid argument"):
        ctx.build_corrections_into(hs, ht, prp, pcol, pvals, inputs_on_host=True, capacity=nnz - 1)
    assert ctx.last_nnz == nnz
    # and the context is still usable
    n, _ = ctx.build_corrections_into(hs, ht, prp, pcol, pvals, inputs_on_host=True)
    assert n == nnz
