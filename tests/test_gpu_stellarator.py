"""The stellarator of Sec. 5 (eq. stellarator, 24 x 72 parameter cells, 3,456 patches):
Green's identity 1/2 u = S[du/dn] - D[u] at every node for u = 1/|x| (harmonic inside;
the origin lies in the hole), evaluated with rrq_apply (smooth direct sum + corrections),
at p = 4, 6, 8: the relative max error must fall with p; and sampled rows against the
oracle."""
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
