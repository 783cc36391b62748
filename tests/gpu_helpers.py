"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np

from oracle import brute

KINDS = ("S", "D", "SP", "DP")
# FP64 path against the FP64 oracle: both follow the same algorithm with different
# operation order, harmonic normalisation and fit solver, so they agree to rounding
# amplified by the fit's condition number (~1e5 at p = 8) and the monomial SSQ basis.
TOL_E = 1e-10


def smooth_part(kind, d, tg, rowptr, col):
    """K(x_t, x_col) w_col for every CSR entry, 0 where the column is the target's node."""
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    k = brute.kernel(kind, tg.xyz[rows], tg.nrm[rows], d.xyz[col], d.nrm[col]) * d.wts[col]
    k[tg.self_node[rows] == col] = 0.0
    return k


def row_error(kind, d, tg, rowptr, col, v_gpu, v_orc):
    """E = max over rows of |row_gpu - row_orc|_inf / |RRQ part of row_orc|_inf."""
    rrq = np.abs(v_orc + smooth_part(kind, d, tg, rowptr, col))
    diff = np.abs(v_gpu - v_orc)
    nrow = len(rowptr) - 1
    num = np.zeros(nrow)
    den = np.zeros(nrow)
    idx = np.repeat(np.arange(nrow), np.diff(rowptr))
    np.maximum.at(num, idx, diff)
    np.maximum.at(den, idx, rrq)
    ok = den > 0
    return float(np.max(num[ok] / den[ok])) if ok.any() else 0.0


def gpu_build(ctx, d, tg, kernels=KINDS, on_host=False, **kw):
    import torch
    from paper_2411_08342_gb300 import rrq
    if on_host:
        arrs = dict(order=d.order, node_off=d.node_off, xyz=d.xyz, nrm=d.nrm, wts=d.wts, txyz=tg.xyz, tnrm=tg.nrm,
                    tself=tg.self_node)
        arrs = {k: np.ascontiguousarray(v) for k, v in arrs.items()}
    else:
        arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    csr = ctx.build_corrections(surf, targ, kernels, inputs_on_host=on_host, **kw)
    rowptr, col, vals = ctx.csr_to_host(csr, kernels)
    diag = ctx.diagnostics()
    ctx.csr_free(csr)
    torch.cuda.synchronize()
    nnz = int(rowptr[-1])
    return rowptr, col[:nnz], {k: v[:nnz] for k, v in vals.items()}, diag
