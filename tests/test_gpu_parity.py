"""CUDA path (through the C ABI) against the CPU FP64 oracle, element by element.

CSR structure (row pointers, columns) must be identical to the FP64 oracle's; values are
gated against the binary128 build of the oracle (E_true <= max(1e-10, 4 x the FP64
oracle's own E_true), see gpu_helpers).  Sizes span several tiles and ragged tails:
orders 2..8 (9..12 in test_gpu_high_order.py), on-surface (self and near) and off-surface targets down to 1e-6 h.
"""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import KINDS, compare_with_oracle as _compare, gpu_build

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


@pytest.mark.parametrize("p", [4, 5])
def test_sphere80_all_rows(ctx, oracle_lib, p):
    """Unit sphere, 80 patches, all on-surface nodes, S D S' D'."""
    d, tg = W.sphere80(p)
    errs, diag = _compare(ctx, oracle_lib, d, tg, label=f"sphere80 p={p}", truth_max=800)
    assert diag["on_edge"] == 0


@pytest.mark.parametrize("p", [2, 3, 6, 7, 8])
def test_orders_on_and_off_surface(ctx, oracle_lib, p):
    d = W.discretize(W.star_surface(2), p)
    rng = np.random.default_rng(p)
    on = W.on_surface_targets(d)
    sel = rng.choice(on.n, min(on.n, 300), replace=False)
    tg = W.concat_targets(W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel]),
                          W.off_surface_targets(d, 300, seed=p))
    _compare(ctx, oracle_lib, d, tg, label=f"star320 p={p}", truth_max=600 if p <= 5 else 200)


def test_star1280_offsurface_p6(ctx, oracle_lib):
    """The star surface (1280 patches, p = 6) with 3000 targets at 10^-k h, k ~ U[0,6]."""
    d, tg = W.star1280(6, 3000)
    _compare(ctx, oracle_lib, d, tg, label="star1280 p=6 3000 targets")


def test_host_inputs_same_as_device(ctx, oracle_lib):
    d, tg = W.sphere80(4)
    a = gpu_build(ctx, d, tg, on_host=False)
    b = gpu_build(ctx, d, tg, on_host=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for k in KINDS:
        assert np.array_equal(a[2][k], b[2][k])


def test_mixed_orders(ctx, oracle_lib):
    """Patches of orders 3, 4, 6 in one surface."""
    base = W.sphere_surface(2)
    rng = np.random.default_rng(0)
    orders = rng.choice([3, 4, 6], base.npatch)
    parts = [W.discretize(base, p) for p in (3, 4, 6)]
    xyz, nrm, wts, node_off = [], [], [], [0]
    for P, p in enumerate(orders):
        dp = parts[[3, 4, 6].index(p)]
        a, b = dp.node_off[P], dp.node_off[P + 1]
        xyz.append(dp.xyz[a:b]); nrm.append(dp.nrm[a:b]); wts.append(dp.wts[a:b])
        node_off.append(node_off[-1] + b - a)
    d = W.Discretization(p=6, npatch=base.npatch, order=orders.astype(np.int32),
                         node_off=np.array(node_off, np.int64), xyz=np.concatenate(xyz), nrm=np.concatenate(nrm),
                         wts=np.concatenate(wts), ref_uv={p: W.ref_nodes(p) for p in (3, 4, 6)}, surface=base)
    on = W.on_surface_targets(d)
    tg = W.concat_targets(on, W.Targets(on.xyz[::7] + 0.01 * on.nrm[::7], on.nrm[::7],
                                        -np.ones(len(on.xyz[::7]), np.int64)))
    _compare(ctx, oracle_lib, d, tg)


def test_edge_cases(ctx, oracle_lib):
    """No targets; targets far from the surface (empty rows); one patch, one target."""
    d, tg = W.sphere80(4)
    empty = W.Targets(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.int64))
    rowptr, col, vals, diag = gpu_build(ctx, d, empty)
    assert rowptr.tolist() == [0] and len(col) == 0
    far = W.Targets(np.array([[10.0, 0, 0], [0, -7.0, 3.0]]), np.array([[1.0, 0, 0], [0, 1.0, 0]]),
                    np.array([-1, -1], np.int64))
    rowptr, col, vals, diag = gpu_build(ctx, d, far)
    assert rowptr.tolist() == [0, 0, 0]
    one = W.discretize(W.flat_surface(np.array([[[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]]])), 5)
    t1 = W.Targets(np.array([[0.3, 0.3, 1e-5]]), np.array([[0, 0, 1.0]]), np.array([-1], np.int64))
    _compare(ctx, oracle_lib, one, t1)


def test_degenerate_patch(ctx):
    """A patch whose nodes are collinear (zero area) is reported, not built: the build
    returns "degenerate patch or singular fit" before any per-pair kernel runs, and the
    fit conditioning of that patch is infinite while its neighbour's is finite."""
    import torch
    from paper_2411_08342_gb300 import rrq
    tris = np.array([[[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]], [[0, 0, 1.0], [1.0, 0, 1.0], [2.0, 0, 1.0]]])
    d = W.discretize(W.flat_surface(tris), 4)
    d.nrm = np.nan_to_num(d.nrm)            # the map has no normal on the degenerate patch
    tg = W.Targets(np.array([[0.3, 0.3, 0.01], [0.2, 0.1, -0.02]]), np.array([[0, 0, 1.0], [0, 0, 1.0]]),
                   np.array([-1, -1], np.int64))
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    with pytest.raises(rrq.RRQError, match="degenerate"):
        ctx.build_corrections(surf, targ)
    k = ctx.fit_condition(surf).cpu().numpy()
    assert np.isfinite(k[0]) and np.isinf(k[1]), k
    torch.cuda.synchronize()
    # the context stays usable
    d2, tg2 = W.sphere80(4)
    assert gpu_build(ctx, d2, tg2)[3]["npairs"] > 0


def test_bad_arguments(ctx):
    from paper_2411_08342_gb300 import rrq
    d, tg = W.sphere80(4)
    bad = d.order.copy()
    bad[3] = 15   # above the largest supported order
    arrs = {k: np.ascontiguousarray(v) for k, v in dict(node_off=d.node_off, xyz=d.xyz, nrm=d.nrm, wts=d.wts).items()}
    surf = ctx.surface(bad, arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(np.ascontiguousarray(tg.xyz), np.ascontiguousarray(tg.nrm), np.ascontiguousarray(tg.self_node))
    with pytest.raises(rrq.RRQError, match="invalid argument"):
        ctx.build_corrections(surf, targ, inputs_on_host=True)


@pytest.mark.parametrize("where", ["node", "normal", "weight", "target", "target_normal"])
def test_nonfinite_inputs_rejected(ctx, where):
    """A NaN (or infinity) in any floating-point input array is an argument error found
    by one device pass before the build, with the array named; the context stays usable."""
    import torch
    from paper_2411_08342_gb300 import rrq
    d, tg = W.sphere80(4)
    a = rrq.device_inputs(d, tg)
    key, idx, val = {"node": ("xyz", 123, float("nan")), "normal": ("nrm", 7, float("nan")),
                     "weight": ("wts", 799, float("inf")), "target": ("txyz", 2, float("nan")),
                     "target_normal": ("tnrm", 2399, float("-inf"))}[where]
    a[key].view(-1)[idx] = val
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    with pytest.raises(rrq.RRQError, match="non-finite"):
        ctx.build_corrections(surf, targ)
    with pytest.raises(rrq.RRQError, match="non-finite"):
        out = {"D": torch.zeros(tg.n, dtype=torch.float64, device="cuda")}
        ctx.evaluate_near(surf, targ, torch.ones(d.nnode, dtype=torch.float64, device="cuda"), out)
    torch.cuda.synchronize()
    d2, tg2 = W.sphere80(4)
    assert gpu_build(ctx, d2, tg2)[3]["npairs"] > 0


def test_full_size_sampled_rows(ctx, oracle_lib):
    """The benchmark workload (star, 1280 patches, p = 6, 200k targets) built in full
    on the GPU, with 200 seeded rows checked against the oracle."""
    d, tg = W.star1280(6, 200_000)
    rng = np.random.default_rng(11)
    tsel = np.sort(rng.choice(tg.n, 200, replace=False))
    errs, diag = _compare(ctx, oracle_lib, d, tg, tsel, label="star1280 p=6 200k targets (benchmark)")
    assert diag["npairs"] > 200_000 * 10


def test_full_size_torus_p8_sampled(ctx, oracle_lib):
    """The wavy-torus workload (20,480 patches, p = 8; 737,280 on-surface nodes and
    200,000 off-surface targets) built in full on the GPU; 60 seeded on-surface and 60
    off-surface rows copied back and checked against the oracle."""
    d, tg = W.wavy_torus()
    non = d.nnode
    rng = np.random.default_rng(12)
    tsel = np.sort(np.concatenate([rng.choice(non, 60, replace=False), non + rng.choice(tg.n - non, 60, replace=False)]))
    errs, diag = _compare(ctx, oracle_lib, d, tg, tsel, sampled=True, label="wavy torus p=8")
    assert diag["npairs"] > 10_000_000


def test_full_size_ellipsoid_sampled(ctx, oracle_lib):
    """The ellipsoid (2, 1, 0.5) on 81,920 patches, p = 6, all 1,720,320 on-surface nodes
    as targets, built in full on the GPU; 100 seeded rows checked against the oracle."""
    d, tg = W.ellipsoid81920()
    rng = np.random.default_rng(13)
    tsel = np.sort(rng.choice(tg.n, 100, replace=False))
    errs, diag = _compare(ctx, oracle_lib, d, tg, tsel, sampled=True, label="ellipsoid 81920 p=6")
    assert diag["npairs"] > 20_000_000


@pytest.mark.parametrize("on_host", [False, True])
def test_apply_correction(ctx, oracle_lib, on_host):
    """rrq_apply_correction: C sigma alone (and accumulated onto out), against numpy on the
    CUDA CSR (the same sums, other order) and on the binary128 oracle's CSR."""
    import torch
    from paper_2411_08342_gb300 import rrq
    from tests.gpu_helpers import truth_csr_rows
    d, tg = W.star1280(6, 1500, seed=41)
    sig = W.random_ylm_density(d.xyz, 6, seed=9)
    arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    csr = ctx.build_corrections(surf, targ)
    rowptr, col, vals = ctx.csr_to_host(csr)
    nnz = int(rowptr[-1])
    sel = np.arange(0, tg.n, 5)
    trp, tcol, tvals = truth_csr_rows(oracle_lib, d, tg, sel)
    try:
        for k in KINDS:
            base = np.random.default_rng(3).standard_normal(tg.n)
            if on_host:
                out = base.copy()
                ctx.apply_correction(csr, k, np.ascontiguousarray(sig), out, accumulate=True, on_host=True)
                got = out - base
            else:
                out = torch.as_tensor(base, device="cuda")
                ctx.apply_correction(csr, k, torch.as_tensor(sig, device="cuda"), out, accumulate=True)
                got = out.cpu().numpy() - base
                out0 = torch.full((tg.n,), 7.0, dtype=torch.float64, device="cuda")
                ctx.apply_correction(csr, k, torch.as_tensor(sig, device="cuda"), out0)
                assert np.allclose(out0.cpu().numpy(), got, rtol=0, atol=1e-12 * np.abs(got).max())
            v = vals[k][:nnz]
            ref = np.zeros(tg.n)
            nz = np.diff(rowptr) > 0
            ref[nz] = np.add.reduceat(v * sig[col[:nnz]], rowptr[:-1][nz])
            scale = np.zeros(tg.n)
            scale[nz] = np.add.reduceat(np.abs(v * sig[col[:nnz]]), rowptr[:-1][nz])
            assert np.max(np.abs(got - ref) - 1e-12 * scale - 1e-12 * np.abs(base)) <= 0, k
            tref = np.add.reduceat(tvals[k] * sig[tcol], trp[:-1])
            tsc = np.add.reduceat(np.abs(tvals[k] * sig[tcol]), trp[:-1])
            print(k, "C sigma vs binary128 rows", f"{np.max(np.abs(got[sel] - tref) / tsc):.1e}")
            assert np.max(np.abs(got[sel] - tref) / tsc) <= 1e-7, k
    finally:
        ctx.csr_free(csr)


def test_apply_matches_reference(ctx, oracle_lib):
    """rrq_apply = smooth direct sum + CSR . sigma, against numpy on the oracle's CSR."""
    import torch
    from paper_2411_08342_gb300 import rrq
    from oracle import brute
    d, tg = W.sphere80(5)
    sig = W.random_ylm_density(d.xyz, 4, seed=3)
    arrs = rrq.device_inputs(d, tg)
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    csr = ctx.build_corrections(surf, targ)
    osf = oracle_lib.OracleSurface(d)
    orp, ocol, ovals, _ = osf.csr_rows(tg)
    sdev = torch.as_tensor(sig, dtype=torch.float64, device="cuda")
    for k in KINDS:
        out = torch.empty(tg.n, dtype=torch.float64, device="cuda")
        ctx.apply(surf, targ, k, csr, sdev, out)
        with np.errstate(divide="ignore", invalid="ignore"):
            K = brute.kernel(k, tg.xyz[:, None], tg.nrm[:, None], d.xyz[None], d.nrm[None])
        K[np.arange(tg.n), tg.self_node] = 0
        ref = K @ (d.wts * sig) + np.add.reduceat(ovals[k] * sig[ocol], orp[:-1])
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), k
    ctx.csr_free(csr)
