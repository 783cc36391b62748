"""The allocation-free entry point rrq_build_corrections_static, called through the C ABI,
against rrq_build_corrections on the same inputs, twice in a row.

The static variant exists for callers that must not allocate device memory during a
call (applications that own all device memory through their own allocator, loops that
forbid allocation after start-up, plug-in hosts with a fixed device footprint).  It
keeps its scratch in one static device array that is reused by every call, so the
second call must give the same result as the first.  This file is collected last so
that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KINDS = ("S", "D", "SP", "DP")


def test_static_matches_allocating_build_twice():
    import torch

    from paper_2411_08342_gb300 import rrq
    from tests.gpu_helpers import TOL_E
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    ctx = rrq.Context(0)
    d, tg = W.sphere80(5)
    tg = W.concat_targets(tg, W.off_surface_targets(d, 400, seed=3))
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    csr = ctx.build_corrections(surf, targ, KINDS)
    ref_rowptr, ref_col, ref_vals = ctx.csr_to_torch(csr, KINDS)
    nnz_ref = csr.nnz
    ctx.csr_free(csr)
    dev = torch.device("cuda", 0)
    cap = nnz_ref + 17
    for call in range(2):
        rowptr = torch.full((tg.n + 1,), -1, dtype=torch.int64, device=dev)
        col = torch.full((cap,), -1, dtype=torch.int32, device=dev)
        vals = {k: torch.full((cap,), float("nan"), dtype=torch.float64, device=dev) for k in KINDS}
        nnz, npairs = ctx.build_corrections_static(surf, targ, rowptr, col, vals, KINDS)
        torch.cuda.synchronize()
        assert nnz == nnz_ref, call
        assert torch.equal(rowptr, ref_rowptr), call
        assert torch.equal(col[:nnz], ref_col), call
        for k in KINDS:
            ref = ref_vals[k]
            err = ((vals[k][:nnz] - ref).abs().max() / ref.abs().max()).item()
            assert err <= TOL_E, (call, k, err)
    # a too small output buffer is refused with the needed size reported
    small = torch.empty(8, dtype=torch.int32, device=dev)
    smallv = {k: torch.empty(8, dtype=torch.float64, device=dev) for k in KINDS}
    with pytest.raises(rrq.RRQError, match="invalid argument"):
        ctx.build_corrections_static(surf, targ, torch.empty(tg.n + 1, dtype=torch.int64, device=dev), small, smallv,
                                     KINDS)
    ctx.close()


def test_static_rejects_problems_beyond_its_scratch():
    import torch

    from paper_2411_08342_gb300 import rrq
    ctx = rrq.Context(0)
    d, tg = W.star1280(6, 1000)        # 1280 patches need more than the static maximum
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    dev = torch.device("cuda", 0)
    with pytest.raises(rrq.RRQError, match="scratch"):
        ctx.build_corrections_static(surf, targ, torch.empty(tg.n + 1, dtype=torch.int64, device=dev),
                                     torch.empty(16, dtype=torch.int32, device=dev),
                                     {k: torch.empty(16, dtype=torch.float64, device=dev) for k in KINDS}, KINDS)
    ctx.close()


def test_static_rejects_mixed_precision():
    """The allocation-free build is FP64 only: a request for the mixed path is refused
    (unsupported option) rather than silently built in FP64."""
    import torch

    from paper_2411_08342_gb300 import rrq
    ctx = rrq.Context(0)
    d, tg = W.sphere80(4)
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    dev = torch.device("cuda", 0)
    rowptr = torch.empty(tg.n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(16, dtype=torch.int32, device=dev)
    vals = {k: torch.empty(16, dtype=torch.float64, device=dev) for k in KINDS}
    arr = (rrq.C.c_void_p * 4)()
    for k in KINDS:
        arr[rrq.KERNEL_SLOT[k]] = vals[k].data_ptr()
    opt = rrq.Options(0, 0, 0.0, 0, 0.0, 1)
    nnz, npairs = rrq.C.c_int64(), rrq.C.c_int64()
    st = ctx.L.rrq_build_corrections_static(ctx.h, rrq.C.byref(surf), rrq.C.byref(targ), 15, rrq.C.byref(opt),
                                            rrq._ptr(rowptr), rrq._ptr(col), arr, 16, rrq.C.byref(nnz),
                                            rrq.C.byref(npairs))
    assert ctx.L.rrq_status_string(st).decode() == "unsupported option"
    assert "FP64 only" in ctx.L.rrq_last_error().decode()
    ctx.close()
