"""Pins of the oracle at orders 13 and 14 (the top of the paper's tables, Sec. 5.3).

* Thm. trianglebasis at p = 13, 14: on a flat triangle the F^{(l,m)} = dH/dz span the
  polynomials of degree <= p-1;
* rows of all four kernels on a flat triangle (binary128 build: binary64 rows of order 14
  lose digits to the fit's conditioning, Sec. 5.1) applied to a polynomial density of
  degree 4, against brute-force layer potentials (the fit is exact for it);
* the quaternion fit of Sec. 5.1's interpolation study keeps converging from p = 12 to 14
  for the analytic density 1/(x^2 + y^2 + 0.5);
* on the unit sphere (80 patches) the corrected D reproduces the Y_2^1 eigenvalue better
  at p = 14 than at p = 12.
"""
import math

import numpy as np
import pytest

from oracle import brute
from paper_2411_08342_gb300 import workloads as W

KINDS = ("S", "D", "SP", "DP")
A = np.array([0.1, -0.2, 0.3])
B = np.array([1.0, 0.1, 0.2])
C = np.array([0.3, 0.8, 0.5])
NU = np.cross(B - A, C - A)
NU /= np.linalg.norm(NU)
E1 = (B - A) / np.linalg.norm(B - A)
E2 = np.cross(NU, E1)


def _mu(u, v):
    return 1 + 0.5 * u - 0.3 * v + u * u * v - 2 * v ** 3 + 0.7 * u ** 4


@pytest.mark.parametrize("p", [13, 14])
def test_flat_triangle_basis_theorem_high_order(oracle_lib, p):
    O = oracle_lib
    rng = np.random.default_rng(p)
    pts = rng.random((2 * p * p, 2)) - 0.5
    F = []
    for (x, y) in pts:
        row = []
        for l in range(1, p + 1):
            for m in range(1, l + 1):
                g, _ = O.grad_hess_S(p, [x, y, 0.0], l, m)
                Hg = math.sqrt(2) * g.imag
                assert abs(Hg[0]) < 1e-12 and abs(Hg[1]) < 1e-12
                row.append(Hg[2])
        F.append(row)
    F = np.array(F)
    F /= np.abs(F).max(0)
    mono = np.array([[x ** a * y ** b for a in range(p) for b in range(p - a)] for (x, y) in pts])
    mono /= np.abs(mono).max(0)
    npn = p * (p + 1) // 2
    s = np.linalg.svd(np.hstack([F, mono]), compute_uv=False)
    # [F mono] has rank n_p: a gap of many orders of magnitude after the n_p-th value
    assert s[npn - 1] / s[0] > 1e-9 and s[npn] / s[0] < 1e-11, (s[npn - 1] / s[0], s[npn] / s[0])


@pytest.mark.parametrize("p", [13, 14])
@pytest.mark.parametrize("where", ["above", "near_edge", "far"])
def test_flat_triangle_rows_high_order(oracle_lib, p, where):
    d = W.discretize(W.flat_surface(np.array([[A, B, C]])), p)
    o128 = oracle_lib.OracleSurface(d, ext=True)
    xt = {"above": (A + B + C) / 3 + 0.1 * E1 + 0.05 * NU,
          "near_edge": (A + B) / 2 + 0.05 * E2 + 0.01 * NU,
          "far": A + 0.3 * (B - A) + 0.4 * NU}[where]
    nt = np.array([0.3, -0.5, 0.8])
    nt /= np.linalg.norm(nt)
    tg = W.Targets(xt[None], nt[None], np.array([-1]))
    vals, _, flags = o128.rows(tg, [0], [0])
    assert flags[0] == 0
    uv = W.ref_nodes(p)
    sig = _mu(uv[:, 0], uv[:, 1])
    for kind in KINDS:
        sm = sum(brute.kernel(kind, xt, nt, d.xyz[i][None], d.nrm[i][None])[0] * d.wts[i] * sig[i]
                 for i in range(len(sig)))
        got = vals[kind] @ sig + sm
        ref = brute.flat_triangle(kind, A, B, C, xt, nt, _mu)
        assert abs(got - ref) < 2e-11 * max(1.0, abs(ref)), (kind, got, ref)


def test_quaternion_interpolation_p14(oracle_lib):
    O = oracle_lib
    R = 1 / np.sqrt(3)
    ang = 0.5 * np.pi + 2 * np.pi * np.arange(3) / 3
    tri = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros(3)], -1)[None]
    rng = np.random.default_rng(0)
    a, b = rng.random(2000), rng.random(2000)
    sw = a + b > 1
    a[sw], b[sw] = 1 - a[sw], 1 - b[sw]
    V = tri[0]
    pts = V[0] + a[:, None] * (V[1] - V[0]) + b[:, None] * (V[2] - V[0])
    f = lambda x, y: 1 / (x * x + y * y + 0.5)
    err = {}
    for p in (12, 14):
        d = W.discretize(W.flat_surface(tri), p)
        info = O.OracleSurface(d, ext=True).patch_internals(0)
        npn = p * (p + 1) // 2
        fr = info["frame"]
        c0, Rm, s = fr[:3], fr[3:12].reshape(3, 3), fr[12]
        XD = info["XD"].reshape(4, npn, npn)
        mu = f(d.xyz[:, 0], d.xyz[:, 1])
        c = np.einsum("qli,i->lq", XD, mu)
        _, gH = O.basis_batch(p, s * (pts - c0) @ Rm)
        q0 = -np.einsum("mla,la->m", gH, c[:, 1:])
        ref = f(pts[:, 0], pts[:, 1])
        err[p] = np.abs(q0 - ref).max() / np.abs(ref).max()
    assert err[14] < err[12] / 3, err


def test_sphere_eigenvalue_p14(oracle_lib):
    """D_pv[Y_2^1] = -Y_2^1 / 10 on the unit sphere: the full operator (smooth rule +
    correction) at 150 nodes of the 80-patch mesh, p = 12 and p = 14."""
    O = oracle_lib
    err = {}
    for p in (12, 14):
        d = W.discretize(W.sphere_surface(1), p)
        on = W.on_surface_targets(d)
        sel = np.random.default_rng(p).choice(on.n, 150, replace=False)
        tg = W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel])
        rowptr, col, vals, _ = O.OracleSurface(d).csr_rows(tg, kernels=("D",))
        Y = W.real_ylm(2, 1, d.xyz)
        with np.errstate(divide="ignore", invalid="ignore"):
            K = brute.kernel("D", tg.xyz[:, None], tg.nrm[:, None], d.xyz[None], d.nrm[None])
        K[np.arange(tg.n), tg.self_node] = 0
        y = K @ (d.wts * Y) + np.add.reduceat(vals["D"] * Y[col], rowptr[:-1])
        err[p] = np.abs(y + Y[tg.self_node] / 10).max() / np.abs(Y).max()
    assert err[14] < err[12] / 3 and err[14] < 2e-9, err
