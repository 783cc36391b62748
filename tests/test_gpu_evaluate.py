"""Density-given near evaluation (rrq_evaluate_near): the correction applied to a density
without storing the matrix (Sec. 4 Steps 1-8 with Step 2).

* Against the CSR of rrq_build_corrections times the same density, up to the different
  summation order (B . (X sigma) against sum_i (B . X_i) sigma_i): per target,
  |difference| <= 1e-12 x sum_j (|C_tj| + |K(t, x_j) w_j|) |sigma_j| over the row (the RRQ
  part and the smooth part it cancels are both summed).
* Against the oracle, independently of the CUDA CSR: C_true sigma with C_true the rows of
  the binary128 oracle, with the same normalisation; the gate is the apply gate of the
  build, max(1e-10, TRUTH_FACTOR x the FP64 oracle's own C sigma error)."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import KINDS, TOL_APPLY, TRUTH_FACTOR, fmt, smooth_part, truth_csr_rows

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


def _cases():
    d5, t5 = W.sphere80(5)
    d6, t6 = W.star1280(6, 3000, seed=31)
    d10 = W.discretize(W.sphere_surface(1), 10)
    return {"sphere80_p5_on": (d5, t5), "star1280_p6_off": (d6, t6),
            "sphere80_p10_on": (d10, W.on_surface_targets(d10))}


@pytest.mark.parametrize("name", ["sphere80_p5_on", "star1280_p6_off", "sphere80_p10_on"])
@pytest.mark.parametrize("on_host", [False, True])
def test_evaluate_near_matches_csr(ctx, name, on_host):
    import torch
    from paper_2411_08342_gb300 import rrq
    d, tg = _cases()[name]
    sig = W.random_ylm_density(d.xyz, 6, seed=5)
    arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    csr = ctx.build_corrections(surf, targ)
    rowptr, col, vals = ctx.csr_to_host(csr)
    ctx.csr_free(csr)
    nnz = int(rowptr[-1])
    col = col[:nnz]
    if on_host:
        h = {k: np.ascontiguousarray(v) for k, v in dict(order=d.order, node_off=d.node_off, xyz=d.xyz, nrm=d.nrm,
                                                         wts=d.wts, txyz=tg.xyz, tnrm=tg.nrm,
                                                         tself=tg.self_node).items()}
        hs = ctx.surface(h["order"], h["node_off"], h["xyz"], h["nrm"], h["wts"], d.ref_uv)
        ht = ctx.targets(h["txyz"], h["tnrm"], h["tself"])
        outs = {k: np.zeros(tg.n) for k in KINDS}
        ctx.evaluate_near(hs, ht, np.ascontiguousarray(sig), outs, inputs_on_host=True)
        got = outs
    else:
        outs = {k: torch.zeros(tg.n, dtype=torch.float64, device="cuda") for k in KINDS}
        ctx.evaluate_near(surf, targ, torch.as_tensor(sig, device="cuda"), outs)
        got = {k: v.cpu().numpy() for k, v in outs.items()}
    diag = ctx.diagnostics()
    assert diag["npairs"] > 0
    for k in KINDS:
        v = vals[k][:nnz]
        ref = np.add.reduceat(v * sig[col], rowptr[:-1])
        sm = smooth_part(k, d, tg, rowptr, col)
        scale = np.add.reduceat((np.abs(v) + np.abs(sm)) * np.abs(sig[col]), rowptr[:-1])
        err = np.max(np.abs(got[k] - ref) / scale)
        print(name, k, f"evaluate_near vs CSR: {err:.1e}")
        assert err <= 1e-12, (k, err)


@pytest.mark.parametrize("name", ["sphere80_p5_on", "star1280_p6_off", "sphere80_p10_on"])
def test_evaluate_near_against_oracle(ctx, oracle_lib, name):
    """evaluate_near against C sigma of the oracle's rows (binary128 truth and FP64), on up
    to 400 seeded targets of each case."""
    import torch
    from paper_2411_08342_gb300 import rrq
    d, tg = _cases()[name]
    sig = W.random_ylm_density(d.xyz, 6, seed=5)
    arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    outs = {k: torch.zeros(tg.n, dtype=torch.float64, device="cuda") for k in KINDS}
    ctx.evaluate_near(surf, targ, torch.as_tensor(sig, device="cuda"), outs)
    got = {k: v.cpu().numpy() for k, v in outs.items()}
    rng = np.random.default_rng(17)
    tsel = np.sort(rng.choice(tg.n, min(tg.n, 400), replace=False))
    sub = W.Targets(tg.xyz[tsel], tg.nrm[tsel], tg.self_node[tsel])
    orp, ocol, ovals, _ = oracle_lib.OracleSurface(d).csr_rows(tg, tsel)
    trp, tcol, tvals = truth_csr_rows(oracle_lib, d, tg, tsel)
    assert np.array_equal(orp, trp) and np.array_equal(ocol, tcol)
    nz = np.diff(orp) > 0
    egpu, eorc = {}, {}
    for k in KINDS:
        sm = smooth_part(k, d, sub, orp, ocol)
        scale = np.zeros(len(tsel))
        ref, o64 = np.zeros(len(tsel)), np.zeros(len(tsel))
        scale[nz] = np.add.reduceat((np.abs(tvals[k]) + np.abs(sm)) * np.abs(sig[ocol]), orp[:-1][nz])
        ref[nz] = np.add.reduceat(tvals[k] * sig[ocol], orp[:-1][nz])
        o64[nz] = np.add.reduceat(ovals[k] * sig[ocol], orp[:-1][nz])
        egpu[k] = float(np.max(np.abs(got[k][tsel] - ref)[nz] / scale[nz]))
        eorc[k] = float(np.max(np.abs(o64 - ref)[nz] / scale[nz]))
        assert np.all(got[k][tsel][~nz] == 0.0), k
    print(name, "evaluate_near vs binary128 C sigma", fmt(egpu), "FP64 oracle C sigma", fmt(eorc))
    for k in KINDS:
        assert egpu[k] <= max(TOL_APPLY, TRUTH_FACTOR * eorc[k]), (k, egpu[k], eorc[k])


def test_evaluate_near_arguments(ctx):
    import torch
    from paper_2411_08342_gb300 import rrq
    d, tg = W.sphere80(4)
    arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    sig = torch.ones(d.nnode, dtype=torch.float64, device="cuda")
    out = {"D": torch.zeros(tg.n, dtype=torch.float64, device="cuda")}
    opt = rrq.Options(0, 0, 0.0, 0, 0.0, 1)
    arr = (rrq.C.c_void_p * 4)()
    arr[1] = out["D"].data_ptr()
    st = ctx.L.rrq_evaluate_near(ctx.h, rrq.C.byref(surf), rrq.C.byref(targ), rrq.D, rrq._ptr(sig), arr,
                                 rrq.C.byref(opt))
    assert ctx.L.rrq_status_string(st).decode() == "unsupported option"
    with pytest.raises(rrq.RRQError, match="invalid argument"):
        ctx.evaluate_near(surf, targ, sig, {})
