"""Conditioning of the density fits on the GPU (rrq_fit_condition, rrq_diag.kappa_max):
kappa_1(A) per patch in the paper's harmonic normalisation (Sec. 5.1) against the
oracle's, which comes from an explicit inverse of the real 4 n_p x 4 n_p block matrix.
The GPU takes ||A||_1 from the harmonic gradients and ||A^{-1}||_1 from the quaternion
solves of the fit.  Both inverses carry rounding errors that grow with kappa; the
tolerance is max(1e-8, 1e-18 kappa) relative (at p = 12, kappa reaches 5e12 on the most
curved paraboloid patch, where the two differ by 6e-7)."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-8


def _tol(k):
    return max(RTOL, 1e-18 * k)


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2411_08342_gb300 import rrq
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    c = rrq.Context(0)
    yield c
    c.close()


def _surface(ctx, d, on_host=False):
    from paper_2411_08342_gb300 import rrq
    if on_host:
        a = {k: np.ascontiguousarray(getattr(d, k)) for k in ("order", "node_off", "xyz", "nrm", "wts")}
    else:
        a = rrq.device_inputs(d, W.on_surface_targets(d))
    return ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv), a


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_kappa_paraboloid(ctx, oracle_lib, p):
    """Single paraboloid patches (eq. paraboloid) over curvatures and sizes."""
    for H, h in ((0.0, 1.0), (1.0, 1.0), (10.0, 1.0), (10.0, 0.125)):
        d = W.discretize(W.paraboloid_patch(H, h), p)
        s, keep = _surface(ctx, d)
        k_gpu = float(ctx.fit_condition(s).cpu()[0])
        k_orc = oracle_lib.OracleSurface(d).patch_kappa(0)
        print(f"p={p} H={H} h={h}: kappa gpu {k_gpu:.6e} oracle {k_orc:.6e}")
        assert abs(k_gpu - k_orc) <= _tol(k_orc) * k_orc, (p, H, h, k_gpu, k_orc)


@pytest.mark.parametrize("on_host", [False, True])
def test_kappa_surfaces_and_diag(ctx, oracle_lib, on_host):
    """Every patch of two curved surfaces (a star at p = 6, a wavy torus at p = 4), with
    host and device buffers; the largest value is what a build reports in
    rrq_diag.kappa_max."""
    d1 = W.discretize(W.star_surface(1), 6)
    d2 = W.discretize(W.wavy_torus_surface(8, 16), 4)
    for d in (d1, d2):
        s, keep = _surface(ctx, d, on_host)
        k = ctx.fit_condition(s, on_host=on_host)
        k = k if on_host else k.cpu().numpy()
        osf = oracle_lib.OracleSurface(d)
        ko = np.array([osf.patch_kappa(P) for P in range(d.npatch)])
        err = np.max(np.abs(k - ko) / ko)
        print(d.surface.name, f"p={d.p} kappa max {ko.max():.3e}, max rel diff {err:.1e}")
        assert err <= RTOL
    # the build's diagnostic: max over the patches of the surface it built
    from tests.gpu_helpers import gpu_build
    _, _, _, diag = gpu_build(ctx, d1, W.off_surface_targets(d1, 200, seed=3))
    ko = max(oracle_lib.OracleSurface(d1).patch_kappa(P) for P in range(d1.npatch))
    assert abs(diag["kappa_max"] - ko) <= RTOL * ko


def test_kappa_batch_diag(ctx, oracle_lib):
    """A batch reports the largest kappa over all its surfaces."""
    items = W.star_batch(3, levels=(1,), orders=(4, 6), seed=W.WORKLOAD_SEED + 60)
    surfs, targs, keep = [], [], []
    from paper_2411_08342_gb300 import rrq
    for d, tg in items:
        a = rrq.device_inputs(d, tg)
        keep.append(a)
        surfs.append(ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv))
        targs.append(ctx.targets(a["txyz"], a["tnrm"], a["tself"]))
    b = ctx.batch(surfs, targs, kernels=("D",))
    try:
        b.execute()
        kmax = ctx.diagnostics()["kappa_max"]
    finally:
        b.close()
    ko = max(oracle_lib.OracleSurface(d).patch_kappa(P) for d, _ in items for P in range(d.npatch))
    assert abs(kmax - ko) <= RTOL * ko
