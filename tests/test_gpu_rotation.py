"""The O(p^3) rotation-based translation of Step 7 (Sec. 2.3, the remark on fast
translation; rrq_options.translation = 1) against the oracle, whose translation is the
direct sum of eqs. l2ltranslation2-3: the two compute the same quantity, so the rows of the
rotation build must meet the same binary128 truth gate as the direct build, at every order,
and on targets where the rotation is degenerate (at the frame origin, rho = 0; on the polar
axis of the harmonics, theta = 0 and pi)."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.gpu_helpers import KINDS, compare_with_oracle, gpu_build

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


def _targets(d, n_on, n_off, seed):
    rng = np.random.default_rng(seed)
    on = W.on_surface_targets(d)
    sel = rng.choice(on.n, min(on.n, n_on), replace=False)
    return W.concat_targets(W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel]),
                            W.off_surface_targets(d, n_off, seed=seed))


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, 10, 12])
def test_rotation_translation_against_oracle(ctx, oracle_lib, p):
    """Star surface of 80 patches, 150 on-surface nodes and 150 targets at 10^-k h, all four
    kernels: rows and applies within the gate of the direct sums."""
    d = W.discretize(W.star_surface(1), p)
    tg = _targets(d, 150, 150, seed=300 + p)
    errs, diag = compare_with_oracle(ctx, oracle_lib, d, tg, truth_max=160, label=f"rotation p={p}", rotation=True)
    assert diag["npairs"] > 0


def test_rotation_order_14_applies(ctx, oracle_lib):
    """p = 14 on the 80-patch sphere, gated on the applies (what a correction does to a
    smooth density).  Rows are printed, not gated: at this order the fit's condition number
    makes the rows of both binary64 forms rounding-dominated (the FP64 oracle's own row
    error is 4e-3 to 2e-2 here), and the rotation form rounds them further, because its
    back rotation carries every component of each degree -- the real parts and the m <= 0
    parts that the rows never use, which are much larger than the imaginary m >= 1 parts
    they do use -- and their rounding spreads into the small ones (measured: S' rows 1.9e-2
    against the oracle's 4.4e-3)."""
    d = W.discretize(W.sphere_surface(1), 14)
    tg = _targets(d, 150, 150, seed=314)
    errs, diag = compare_with_oracle(ctx, oracle_lib, d, tg, truth_max=160, label="rotation p=14", gate_rows=False,
                                     rotation=True)
    assert diag["npairs"] > 0


@pytest.mark.parametrize("p", [4, 9])
def test_rotation_degenerate_angles(ctx, oracle_lib, p):
    """Targets at the frame origin of a patch (the vertex mean: rho = 0), and on the line
    through it along the frame's e_x, the polar axis of the harmonics S (theta = 0 and pi),
    plus along e_z (theta = pi / 2), with random unit normals, for 12 patches."""
    d = W.discretize(W.star_surface(1), p)
    osf = oracle_lib.OracleSurface(d)
    rng = np.random.default_rng(11 + p)
    pts = []
    for P in rng.choice(len(d.order), 12, replace=False):
        fr = osf.patch_internals(int(P))
        c, R, s = fr["c"], fr["R"], fr["s"]
        L = 1.0 / s
        pts += [c, c + 0.3 * L * R[:, 0], c - 0.3 * L * R[:, 0], c + 0.2 * L * R[:, 2], c - 0.2 * L * R[:, 2]]
    xyz = np.array(pts)
    nrm = rng.normal(size=xyz.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    tg = W.Targets(xyz, nrm, -np.ones(len(xyz), np.int64))
    errs, diag = compare_with_oracle(ctx, oracle_lib, d, tg, label=f"rotation, degenerate angles p={p}",
                                     rotation=True)
    assert diag["npairs"] >= len(xyz)


def test_rotation_equals_direct_to_rounding(ctx):
    """Sphere of 80 patches at p = 8: the applies of the rotation build and of the direct
    build to a smooth density agree to 1e-12.  Their rows differ by the rounding of the two
    forms, amplified like every row error by the fit (measured: up to 9.4e-9 of a row's
    largest entry, printed; on the 80-patch star at p = 8 the rows of either form lie
    1e-8 to 4e-8 from the binary128 truth)."""
    d = W.discretize(W.sphere_surface(1), 8)
    tg = _targets(d, 400, 300, seed=5)
    rp, col, v_dir, _ = gpu_build(ctx, d, tg, KINDS)
    rp2, col2, v_rot, _ = gpu_build(ctx, d, tg, KINDS, rotation=True)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    sigma = W.random_ylm_density(d.xyz, 8, seed=3)
    lens = np.diff(rp)
    full = np.nonzero(lens)[0]
    rows = np.repeat(np.arange(tg.n), lens)
    worst = {}
    for k in KINDS:
        rowmax = np.maximum.reduceat(np.abs(v_dir[k]), rp[full])
        scale = np.repeat(rowmax, lens[full])
        worst[k] = float(np.max(np.abs(v_rot[k] - v_dir[k]) / scale))
        a_dir = np.bincount(rows, weights=v_dir[k] * sigma[col], minlength=tg.n)
        a_rot = np.bincount(rows, weights=v_rot[k] * sigma[col], minlength=tg.n)
        ea = np.abs(a_rot - a_dir).max() / np.abs(a_dir).max()
        assert ea < 1e-12, (k, ea)
    print("rotation vs direct, worst entry relative to its row", {k: f"{v:.1e}" for k, v in worst.items()})


def test_rotation_option_rejected_where_not_built(ctx):
    """translation = 1 is for FP64 matrix builds: with the mixed path, in the evaluation, the
    batch and the allocation-free build it is refused (unsupported option), and a value
    other than 0 and 1 is an invalid argument."""
    import ctypes as C

    import torch
    from paper_2411_08342_gb300 import rrq
    d = W.discretize(W.sphere_surface(1), 4)
    tg = W.on_surface_targets(d)
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    L = ctx.L

    def status(st):
        return L.rrq_status_string(st).decode()

    out = rrq.CSR()
    for prec, tr, want in ((1, 1, "unsupported option"), (0, 2, "invalid argument"), (0, -1, "invalid argument")):
        opt = rrq.Options(0, 0, 0.0, 0, 0.0, prec, tr)
        st = L.rrq_build_corrections(ctx.h, C.byref(surf), C.byref(targ), 15, C.byref(opt), C.byref(out))
        assert status(st) == want, (prec, tr, status(st))
    opt = rrq.Options(0, 0, 0.0, 0, 0.0, 0, 1)
    dens = torch.zeros(len(d.xyz), dtype=torch.float64, device="cuda")
    res = torch.zeros(tg.n, dtype=torch.float64, device="cuda")
    arr = (C.c_void_p * 4)(res.data_ptr(), None, None, None)
    st = L.rrq_evaluate_near(ctx.h, C.byref(surf), C.byref(targ), 1, rrq._ptr(dens), arr, C.byref(opt))
    assert status(st) == "unsupported option"
    dev = torch.device("cuda", 0)
    rowptr = torch.empty(tg.n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(16, dtype=torch.int32, device=dev)
    vals = torch.empty(16, dtype=torch.float64, device=dev)
    varr = (C.c_void_p * 4)(vals.data_ptr(), None, None, None)
    nnz, npairs = C.c_int64(), C.c_int64()
    st = L.rrq_build_corrections_static(ctx.h, C.byref(surf), C.byref(targ), 1, C.byref(opt), rrq._ptr(rowptr),
                                        rrq._ptr(col), varr, 16, C.byref(nnz), C.byref(npairs))
    assert status(st) == "unsupported option"
    surfs, targs = (rrq.Surface * 1)(surf), (rrq.TargetsS * 1)(targ)
    bh = C.c_void_p()
    st = L.rrq_batch_create(ctx.h, 1, surfs, targs, 15, C.byref(opt), 0, C.byref(bh))
    assert status(st) == "unsupported option" and not bh.value
    torch.cuda.synchronize()
