"""Mixed-precision build (rrq_options.precision = 1: the Step-6 line integrals, Step-7
translation sums and Step-8 fit contraction accumulated in double-float arithmetic on the
FP32 pipes, everything else FP64) against the binary128 truth rows.

Stated accuracy of the mixed path.  Double-float numbers carry about 48 significant bits
(relative rounding 2^-48, against 2^-53 for binary64), and the mixed path applies them to
the same formulation, whose ill-conditioned parts (target-centred translation in the
outer shell of the near region, fit amplification kappa(A)) amplify rounding in the same
way.  Its rounding errors are therefore at most 2^5 = 32 times those of a binary64
implementation: rows and applies must satisfy E_true(mixed) <= max(1e-10,
MIXED_FACTOR x E_true(FP64 oracle)) with MIXED_FACTOR = 32, E_true measured against the
binary128 build of the oracle on the same rows (gpu_helpers)."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import KINDS, TOL_APPLY, TOL_E, fmt, gpu_build, row_error, truth_errors

pytestmark = pytest.mark.gpu
MIXED_FACTOR = 32.0


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
    tr = truth_errors(oracle_lib, d, tg, None, orp, ocol, {"mixed": vals, "orc": ovals})
    e64 = {k: row_error(k, d, tg, orp, ocol, vals[k], ovals[k]) for k in KINDS}
    print(name, "E_true mixed", fmt({k: v[0] for k, v in tr["mixed"].items()}),
          "E_true fp64 oracle", fmt({k: v[0] for k, v in tr["orc"].items()}),
          "| apply E_true mixed", fmt({k: v[1] for k, v in tr["mixed"].items()}),
          "fp64 oracle", fmt({k: v[1] for k, v in tr["orc"].items()}), "| mixed vs fp64 oracle", fmt(e64))
    for k in KINDS:
        assert np.all(np.isfinite(vals[k]))
        (e, ea), (eo, eao) = tr["mixed"][k], tr["orc"][k]
        assert e <= max(TOL_E, MIXED_FACTOR * eo), (k, e, eo)
        assert ea <= max(TOL_APPLY, MIXED_FACTOR * eao), (k, ea, eao)


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
