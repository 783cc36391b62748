"""Mixed-precision build (rrq_options.precision = 1: Step-6 line integrals accumulated in
double-float FP32 arithmetic, everything else FP64) against the FP64 oracle.

Stated tolerance of the mixed path: the apply-level gate of the FP64 path unchanged
(max(1e-10, 8 x the oracle's own sensitivity)), and rows within 32 x the oracle's own
rounding sensitivity (measured on the same rows with rigidly rotated inputs) or 1e-10.
Double-float carries ~48 bits, so rows move by a few times more than in FP64 where the
formulation is ill-conditioned (outer shell of the near region); smooth-density applies
do not see it up to order 8.  From order 9 the fit's conditioning (kappa ~ 1e7-1e9 on
these meshes) carries the ~1e-14 relative error of the double-float line integrals into
the applied result at the 1e-10 to 1e-9 level (at p = 10 on the 320-patch star: 2.3e-10
for S, 1.9e-10 for D, 6.5e-10 for S', 1.5e-9 for the hypersingular D'): there the stated
apply tolerance of the mixed path is 5e-9."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import (KINDS, ROT_FACTOR, TOL_APPLY, TOL_E, apply_error, gpu_build, rotated,
                               row_error)

pytestmark = pytest.mark.gpu
MIXED_ROW_FACTOR = 32.0
MIXED_APPLY_TOL_HIGH_ORDER = 5e-9


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
    d8 = W.discretize(W.star_surface(2), 8)
    rng = np.random.default_rng(8)
    on = W.on_surface_targets(d8)
    sel = rng.choice(on.n, 300, replace=False)
    t8 = W.concat_targets(W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel]), W.off_surface_targets(d8, 300, seed=8))
    d10 = W.discretize(W.star_surface(2), 10)
    rng = np.random.default_rng(10)
    on = W.on_surface_targets(d10)
    sel = rng.choice(on.n, 200, replace=False)
    t10 = W.concat_targets(W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel]),
                           W.off_surface_targets(d10, 200, seed=10))
    return {"star1280_p6": W.star1280(6, 600), "star320_p8": (d8, t8), "star320_p10": (d10, t10)}


@pytest.mark.parametrize("name", ["star1280_p6", "star320_p8", "star320_p10"])
def test_mixed_against_oracle(ctx, oracle_lib, name):
    d, tg = _cases()[name]
    rowptr, col, vals, diag = gpu_build(ctx, d, tg, mixed=True)
    orp, ocol, ovals, _ = oracle_lib.OracleSurface(d).csr_rows(tg)
    assert np.array_equal(rowptr, orp) and np.array_equal(col, ocol)
    d2, tg2 = rotated(d, tg)
    _, _, rvals, _ = oracle_lib.OracleSurface(d2).csr_rows(tg2)
    sigma = W.random_ylm_density(d.xyz, 8, seed=7)
    for k in KINDS:
        assert np.all(np.isfinite(vals[k]))
        e = row_error(k, d, tg, orp, ocol, vals[k], ovals[k])
        er = row_error(k, d, tg, orp, ocol, rvals[k], ovals[k])
        ea = apply_error(k, d, tg, orp, ocol, vals[k], ovals[k], sigma)
        era = apply_error(k, d, tg, orp, ocol, rvals[k], ovals[k], sigma)
        print(name, k, f"row {e:.1e} (oracle self {er:.1e}) apply {ea:.1e} (oracle self {era:.1e})")
        assert e <= max(TOL_E, MIXED_ROW_FACTOR * er), (k, e, er)
        tol_apply = TOL_APPLY if d.p <= 8 else MIXED_APPLY_TOL_HIGH_ORDER
        assert ea <= max(tol_apply, ROT_FACTOR * era), (k, ea, era)


def test_mixed_apply_direct_sum(ctx):
    """rrq_apply with precision = 1: smooth terms of sources at least r_c from the target
    in FP32 (hi/lo coordinates, compensated tile sums), closer ones (all in the target's
    CSR row) in FP64 with the correction.  Stated tolerance: per target,
    |apply_mixed - apply_fp64| <= 1e-6 x (sum_j |K(t, x_j) w_j sigma_j| + sum_j |C_tj sigma_j|),
    for off-surface targets down to 1e-6 h and all four kernels."""
    import torch
    from paper_2411_08342_gb300 import rrq
    from oracle import brute
    d, tg = W.star1280(6, 2000, seed=21)
    sig = W.random_ylm_density(d.xyz, 8, seed=4)
    arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    csr = ctx.build_corrections(surf, targ)
    rowptr, col, vals = ctx.csr_to_host(csr)
    sdev = torch.as_tensor(sig, dtype=torch.float64, device="cuda")
    try:
        for k in KINDS:
            o64 = torch.empty(tg.n, dtype=torch.float64, device="cuda")
            o32 = torch.empty_like(o64)
            ctx.apply(surf, targ, k, csr, sdev, o64)
            ctx.apply(surf, targ, k, csr, sdev, o32, mixed=True)
            with np.errstate(divide="ignore", invalid="ignore"):
                K = brute.kernel(k, tg.xyz[:, None], tg.nrm[:, None], d.xyz[None], d.nrm[None])
            nnz = int(rowptr[-1])
            ca = np.add.reduceat(np.abs(vals[k][:nnz] * sig[col[:nnz]]), rowptr[:-1])
            scale = np.abs(K) @ np.abs(d.wts * sig) + ca
            g64, g32 = o64.cpu().numpy(), o32.cpu().numpy()
            err = np.max(np.abs(g32 - g64) / scale)
            print(k, f"mixed apply rel. error {err:.1e} (plain {np.abs(g32 - g64).max() / np.abs(g64).max():.1e})")
            assert err <= 1e-6, (k, err)
        with pytest.raises(rrq.RRQError, match="invalid argument"):
            ctx.apply(surf, targ, "S", None, sdev, o32, mixed=True)
    finally:
        ctx.csr_free(csr)
