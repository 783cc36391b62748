"""Batched build (rrq_batch_*): many surfaces of different sizes and orders in one plan
whose value computation is one CUDA graph.  Every surface's rows must equal the rows
of its own rrq_build_corrections (same kernels, same per-pair arithmetic), and through
that the oracle; one surface is also checked against the oracle directly."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import KINDS, TOL_E, TRUTH_FACTOR, fmt, gpu_build, row_error, truth_errors

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


def _batch_inputs():
    """Six seeded star surfaces (80 or 320 patches; orders 4, 4, 6, 4, 6, 8; on-surface
    nodes as targets), plus a sphere of order 5 with off-surface targets only and a star
    of order 3 with no targets at all."""
    items = W.star_batch(6, levels=(1, 2), seed=W.WORKLOAD_SEED + 50)
    d = W.discretize(W.sphere_surface(1), 5)
    items.append((d, W.off_surface_targets(d, 700, seed=11)))
    d = W.discretize(W.star_surface(1), 3)
    items.append((d, W.Targets(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.int64))))
    return items


@pytest.fixture(scope="module")
def batch_data():
    return _batch_inputs()


def _surf_targ(ctx, d, tg):
    from paper_2411_08342_gb300 import rrq
    a = rrq.device_inputs(d, tg)
    return (ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv),
            ctx.targets(a["txyz"], a["tnrm"], a["tself"]))


def _view_host(ctx, b, s):
    rowptr, col, vals = ctx.csr_to_host(b.view(s))
    nnz = int(rowptr[-1])
    return rowptr, col[:nnz], {k: v[:nnz] for k, v in vals.items()}


@pytest.mark.parametrize("mixed,autotune", [(False, False), (False, True), (True, False)])
def test_batch_equals_single_builds(ctx, batch_data, mixed, autotune):
    st = [_surf_targ(ctx, d, tg) for d, tg in batch_data]
    b = ctx.batch([s for s, _ in st], [t for _, t in st], mixed=mixed, autotune=autotune)
    try:
        info = b.info()
        assert info["nsurf"] == len(batch_data)
        assert info["nrows"] == sum(tg.n for _, tg in batch_data)
        assert info["graph_kernels"] > 0
        for p in (3, 4, 5, 6, 8):
            assert info["tile"][p] > 0
        b.execute()
        first = [_view_host(ctx, b, s) for s in range(len(batch_data))]
        b.execute()
        total_pairs = 0
        for s, (d, tg) in enumerate(batch_data):
            rowptr, col, vals = _view_host(ctx, b, s)
            # executing again recomputes the same values
            assert np.array_equal(rowptr, first[s][0]) and np.array_equal(col, first[s][1])
            for k in KINDS:
                assert np.array_equal(vals[k], first[s][2][k]), (s, k)
            srp, scol, svals, sdiag = gpu_build(ctx, d, tg, mixed=mixed)
            total_pairs += sdiag["npairs"]
            assert np.array_equal(rowptr, srp), f"surface {s}: row pointers"
            assert np.array_equal(col, scol), f"surface {s}: columns"
            for k in KINDS:
                diff = np.abs(vals[k] - svals[k]).max() if len(col) else 0.0
                assert diff == 0.0, f"surface {s} kernel {k}: max |batch - single| = {diff:.3e}"
        assert info["npairs"] == total_pairs
        print("batch", {k: info[k] for k in ("nrows", "nnz", "npairs", "graph_kernels")},
              "tiles", info["tile"], "persistent", info["persistent"], f"autotune {info['ms_autotune']:.1f} ms")
    finally:
        b.close()


def test_batch_against_oracle(ctx, oracle_lib, batch_data):
    """Surfaces 2 (80 strongly curved patches, order 6) and 4 (320 patches, order 6) of the
    batch, on-surface nodes, row by row against the oracle.  On the 80-patch surface the
    edges are curved enough that a straight-chord estimate of the edge root misjudges the
    rule; the rows agree only because the root-finding skips Newton solely where a bound
    excludes a root from the singularity-swap ellipse."""
    st = [_surf_targ(ctx, d, tg) for d, tg in batch_data]
    b = ctx.batch([s for s, _ in st], [t for _, t in st])
    try:
        b.execute()
        got = {s: _view_host(ctx, b, s) for s in (2, 4)}
    finally:
        b.close()
    for s in (2, 4):
        d, tg = batch_data[s]
        assert d.p == 6 and d.npatch == (80 if s == 2 else 320)
        rowptr, col, vals = got[s]
        osf = oracle_lib.OracleSurface(d)
        orp, ocol, ovals, _ = osf.csr_rows(tg, kernels=KINDS)
        assert np.array_equal(rowptr, orp) and np.array_equal(col, ocol)
        tr = truth_errors(oracle_lib, d, tg, None, orp, ocol, {"gpu": vals, "orc": ovals})
        e64 = {k: row_error(k, d, tg, orp, ocol, vals[k], ovals[k]) for k in KINDS}
        print(f"surface {s}: E_true gpu", fmt({k: v[0] for k, v in tr["gpu"].items()}),
              "E_true fp64 oracle", fmt({k: v[0] for k, v in tr["orc"].items()}), "gpu vs fp64 oracle", fmt(e64))
        for k in KINDS:
            assert tr["gpu"][k][0] <= max(TOL_E, TRUTH_FACTOR * tr["orc"][k][0]), (s, k, tr["gpu"][k], tr["orc"][k])


def test_batch_view_apply_and_errors(ctx, batch_data):
    import torch
    from paper_2411_08342_gb300 import rrq
    st = [_surf_targ(ctx, d, tg) for d, tg in batch_data]
    b = ctx.batch([s for s, _ in st], [t for _, t in st], kernels=("D",))
    try:
        b.execute()
        d, tg = batch_data[1]
        sig = torch.as_tensor(W.random_ylm_density(d.xyz, 6, seed=3), device="cuda")
        out_b = torch.empty(tg.n, dtype=torch.float64, device="cuda")
        ctx.apply(st[1][0], st[1][1], "D", b.view(1), sig, out_b)
        single = ctx.build_corrections(st[1][0], st[1][1], ("D",))
        out_s = torch.empty_like(out_b)
        ctx.apply(st[1][0], st[1][1], "D", single, sig, out_s)
        ctx.csr_free(single)
        assert torch.equal(out_b, out_s)
        # a view is not owned by the caller
        with pytest.raises(rrq.RRQError, match="invalid argument"):
            ctx.csr_free(b.view(1))
        with pytest.raises(rrq.RRQError, match="invalid argument"):
            b.view(len(batch_data))
    finally:
        b.close()
    # different reference nodes for one order are rejected
    d, tg = batch_data[0]
    p = d.p
    bad = {p: d.ref_uv[p] * 0.999 + 0.0003}
    from paper_2411_08342_gb300 import rrq as R
    a = R.device_inputs(d, tg)
    s2 = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], bad)
    with pytest.raises(R.RRQError, match="invalid argument"):
        ctx.batch([st[0][0], s2], [st[0][1], st[0][1]])


def test_autotune_keeps_values(batch_data):
    """rrq_autotune changes only the launch shape of later builds on the context."""
    from paper_2411_08342_gb300 import rrq
    c = rrq.Context(0)
    try:
        d, tg = batch_data[4]
        before = gpu_build(c, d, tg)
        surf, targ = _surf_targ(c, d, tg)
        c.autotune(surf, targ)
        after = gpu_build(c, d, tg)
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        for k in KINDS:
            assert np.array_equal(before[2][k], after[2][k]), k
    finally:
        c.close()
