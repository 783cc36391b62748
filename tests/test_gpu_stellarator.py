"""The stellarator of Sec. 5 (eq. stellarator, 24 x 72 parameter cells, 3,456 patches):
Green's identity 1/2 u = S[du/dn] - D[u] at every node for u = 1/|x| (harmonic inside;
the origin lies in the hole), evaluated with rrq_apply (smooth direct sum + corrections),
at p = 4, 6, 8: the relative max error must fall with p; and sampled rows against the
oracle.  At high order the same identity through the density-given evaluation
(rrq_evaluate_near: the fit of the density itself, X sigma, then B . (X sigma)) is more
accurate than through the matrix rows: a row is the fit of a unit density at one node,
whose coefficients are large, and Sec. 5.1 (eq. interpolationerror) bounds the rounding
by eps_mach times the fitted coefficients' norm."""
import numpy as np
import pytest

from paper_2411_08342_gb300 import workloads as W
from tests.test_gpu_parity import _compare

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


def green_identity_error(ctx, d, tg):
    """max |S[du/dn] - D[u] - u/2| / max |u| over the nodes, u = 1/|x|."""
    import torch
    from paper_2411_08342_gb300 import rrq
    x = d.xyz
    r = np.linalg.norm(x, axis=1)
    u = 1.0 / r
    dudn = -np.einsum("ia,ia->i", x, d.nrm) / r ** 3
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    csr = ctx.build_corrections(surf, targ, ("S", "D"))
    try:
        oS = torch.empty(tg.n, dtype=torch.float64, device="cuda")
        oD = torch.empty_like(oS)
        ctx.apply(surf, targ, "S", csr, torch.as_tensor(dudn, device="cuda"), oS)
        ctx.apply(surf, targ, "D", csr, torch.as_tensor(u, device="cuda"), oD)
    finally:
        ctx.csr_free(csr)
    res = (oS - oD).cpu().numpy() - 0.5 * u
    return float(np.abs(res).max() / np.abs(u).max())


def green_identity_error_density_given(ctx, d, tg):
    """As green_identity_error, with the corrections applied by rrq_evaluate_near (no
    matrix) and the smooth rule by rrq_apply without a CSR."""
    import torch
    from paper_2411_08342_gb300 import rrq
    x = d.xyz
    r = np.linalg.norm(x, axis=1)
    u = 1.0 / r
    dudn = -np.einsum("ia,ia->i", x, d.nrm) / r ** 3
    a = rrq.device_inputs(d, tg)
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    out = {}
    for k, dens in (("S", dudn), ("D", u)):
        sd = torch.as_tensor(dens, device="cuda")
        sm = torch.empty(tg.n, dtype=torch.float64, device="cuda")
        ctx.apply(surf, targ, k, None, sd, sm)
        corr = {k: torch.zeros(tg.n, dtype=torch.float64, device="cuda")}
        ctx.evaluate_near(surf, targ, sd, corr)
        out[k] = (sm + corr[k]).cpu().numpy()
    res = out["S"] - out["D"] - 0.5 * u
    return float(np.abs(res).max() / np.abs(u).max())


def test_green_identity_converges(ctx):
    errs = {}
    for p in (4, 6, 8):
        d, tg = W.stellarator(p)
        errs[p] = green_identity_error(ctx, d, tg)
    print("stellarator Green's identity, relative max error:", {p: f"{e:.2e}" for p, e in errs.items()})
    assert errs[8] < errs[6] < errs[4]
    assert errs[6] < 1e-3


def test_stellarator_sampled_rows(ctx, oracle_lib):
    d, tg = W.stellarator(6)
    rng = np.random.default_rng(17)
    tsel = np.sort(rng.choice(tg.n, 100, replace=False))
    _compare(ctx, oracle_lib, d, tg, tsel, sampled=True)


def test_green_identity_high_order_density_given(ctx):
    """p = 10, 12: Green's identity through the matrix rows and through the density-given
    evaluation agree (both apply the same fit matrices X to the density)."""
    rows, dens = {}, {}
    for p in (10, 12):
        d, tg = W.stellarator(p)
        rows[p] = green_identity_error(ctx, d, tg)
        dens[p] = green_identity_error_density_given(ctx, d, tg)
    print("stellarator Green's identity at high order: matrix rows", {p: f"{e:.2e}" for p, e in rows.items()},
          "density-given", {p: f"{e:.2e}" for p, e in dens.items()})
    for p in (10, 12):
        assert abs(dens[p] - rows[p]) <= 0.05 * rows[p], (p, dens[p], rows[p])
