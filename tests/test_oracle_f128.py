"""Pins of the oracle's binary128 build (rrq_oracle.c compiled with -DORC_F128).

That build computes the same algorithm as the FP64 oracle with a rounding unit of
2^-113 and is the truth reference of the GPU accuracy tests.  These pins check it
against values fixed by mathematics, computed here with mpmath at 30+ digits, in cases
where the binary64 build is visibly less accurate, so that a quantity left in binary64
anywhere inside the binary128 build (a constant, a table, a library call) fails them:

* Gauss-Legendre nodes and weights equal the mpmath ones rounded to binary64;
* singularity-swap weights (Sec. 2.4, Sec. 3.4: moments by recurrence, V^T lambda = I)
  at 24 and 28 nodes integrate f(t)/((t-a)^2+b^2)^{m/2} to 1e-15, where cond(V) ~ 1e8-1e10;
* regular solid harmonics R_l^m (eqs. ylmdef, rlmdef) at degree 16 equal the closed
  form from the associated Legendre functions;
* correction rows of all four kernels on a flat triangle of order 8 (Sec. 4 Steps 1-8)
  applied to a polynomial density of degree 4 -- a case where the fit is exact, so the
  RRQ value is the layer potential itself up to the edge quadrature error, which the
  choice of 32 Gauss nodes per edge puts below 1e-18 for these targets -- equal the
  layer potentials integrated by mpmath to 2e-15 of their magnitude; the binary64
  build is off by ~4e-14 there (translation cancellation);
* on the unit sphere the binary128 rows agree with the binary64 rows to binary64 rounding.
"""
import math

import numpy as np
import pytest

from oracle import brute
from paper_2411_08342_gb300 import workloads as W

mp = pytest.importorskip("mpmath")

KINDS = ("S", "D", "SP", "DP")


@pytest.fixture(scope="module")
def O(oracle_lib):
    oracle_lib.lib(ext=True)
    return oracle_lib


def _mp_gauss_legendre(n):
    x0, _ = np.polynomial.legendre.leggauss(n)
    xs, ws = [], []
    for t in x0:
        t = mp.mpf(float(t))
        for _ in range(8):
            t -= mp.legendre(n, t) / mp.diff(lambda s: mp.legendre(n, s), t)
        dp = mp.diff(lambda s: mp.legendre(n, s), t)
        xs.append(t)
        ws.append(2 / ((1 - t * t) * dp * dp))
    return xs, ws


def test_f128_gauss_legendre(O):
    with mp.workdps(40):
        for n in (7, 16, 32):
            x, w = O.gauss_legendre(n, ext=True)
            xm, wm = _mp_gauss_legendre(n)
            for i in range(n):
                assert x[i] == float(xm[i]), (n, i, x[i], xm[i])
                assert w[i] == float(wm[i]), (n, i, w[i], wm[i])


@pytest.mark.parametrize("ab", [(0.2, 0.05), (-0.7, 0.3), (0.95, 0.01)])
def test_f128_ssq_weights(O, ab):
    a, b = ab
    with mp.workdps(34):
        f = lambda t: mp.exp(t) * mp.cos(2 * t)
        am, bm = mp.mpf(a), mp.mpf(b)
        lo, hi = mp.asinh((-1 - am) / bm), mp.asinh((1 - am) / bm)
        r1 = mp.quad(lambda s: f(am + bm * mp.sinh(s)), mp.linspace(lo, hi, 9))
        r3 = mp.quad(lambda s: f(am + bm * mp.sinh(s)) / (bm * mp.cosh(s)) ** 2, mp.linspace(lo, hi, 9))
        for pt in (24, 28):
            xm, _ = _mp_gauss_legendre(pt)
            fx = [f(t) for t in xm]
            l1, l3 = O.ssq_weights(pt, a, b, ext=True)
            s1 = mp.fsum(mp.mpf(float(l1[q])) * fx[q] for q in range(pt))
            s3 = mp.fsum(mp.mpf(float(l3[q])) * fx[q] for q in range(pt))
            # the weights themselves are rounded to binary64: sum_q |l_q f_q| 2^-53 bounds that part
            e1 = 2 * sum(abs(float(l1[q]) * float(fx[q])) for q in range(pt)) * 2.0 ** -53
            e3 = 2 * sum(abs(float(l3[q]) * float(fx[q])) for q in range(pt)) * 2.0 ** -53
            assert abs(s1 - r1) <= max(1e-15 * abs(r1), e1), (pt, float(s1), float(r1))
            assert abs(s3 - r3) <= max(1e-15 * abs(r3), e3), (pt, float(s3), float(r3))


def test_f128_solid_harmonics(O):
    """R_l^m(x) = sqrt((l-m)!/(l+m)!) r^l P_l^m(cos th) e^{i m phi} with the phase of the
    recurrence (eq. associatelegendrerecurrence, Condon-Shortley factor included)."""
    L = 16
    y = np.array([1.7, -2.3, 0.9])
    got = O.solid_R(L, y, ext=True)
    with mp.workdps(40):
        X, Y, Z = (mp.mpf(float(v)) for v in y)
        r = mp.sqrt(X * X + Y * Y + Z * Z)
        ct, phi = Z / r, mp.atan2(Y, X)
        for l in range(L + 1):
            for m in range(0, l + 1):
                ref = mp.sqrt(mp.factorial(l - m) / mp.factorial(l + m)) * r ** l * mp.legenp(l, m, ct) \
                    * mp.expj(m * phi)
                g = got[l * l + l + m]
                scale = float(abs(ref)) + float(r ** l) * 1e-30
                assert abs(g.real - float(ref.real)) <= 4e-16 * scale, (l, m)
                assert abs(g.imag - float(ref.imag)) <= 4e-16 * scale, (l, m)


A = np.array([0.1, -0.2, 0.3])
B = np.array([1.0, 0.1, 0.2])
C = np.array([0.3, 0.8, 0.5])


def _mu(u, v):
    return 1 + 0.5 * u - 0.3 * v + u * u * v - 2 * v ** 3 + 0.7 * u ** 4


def _exact(kind, xt, nt):
    """The layer potential of kind of the density _mu on the triangle ABC at xt (mpmath)."""
    a, b, c = ([mp.mpf(float(v)) for v in P] for P in (A, B, C))
    ab = [b[i] - a[i] for i in range(3)]
    ac = [c[i] - a[i] for i in range(3)]
    n = [ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0]]
    J = mp.sqrt(sum(v * v for v in n))
    n = [v / J for v in n]
    X = [mp.mpf(float(v)) for v in xt]
    T = [mp.mpf(float(v)) for v in nt]

    def f(s, t):
        u, v = s, (1 - s) * t
        d = [X[i] - (a[i] + u * ab[i] + v * ac[i]) for i in range(3)]
        r2 = sum(q * q for q in d)
        rr = mp.sqrt(r2)
        dn = sum(d[i] * n[i] for i in range(3))
        dt = sum(d[i] * T[i] for i in range(3))
        k = {"S": lambda: 1 / rr, "D": lambda: dn / (r2 * rr), "SP": lambda: -dt / (r2 * rr),
             "DP": lambda: sum(n[i] * T[i] for i in range(3)) / (r2 * rr) - 3 * dn * dt / (r2 * r2 * rr)}[kind]()
        return k * _mu(u, v) * (1 - s) * J / (4 * mp.pi)
    return mp.quad(f, [0, 1], [0, 1])


@pytest.mark.parametrize("dist", [0.8, 1.5])
def test_f128_flat_triangle_rows_exact(O, dist):
    p = 8
    d = W.discretize(W.flat_surface(np.array([[A, B, C]])), p)
    o128 = O.OracleSurface(d, ptilde=32, ext=True)
    rng = np.random.default_rng(int(dist * 10))
    cen = (A + B + C) / 3
    L = max(np.linalg.norm(B - A), np.linalg.norm(C - B), np.linalg.norm(A - C))
    dirv = rng.standard_normal(3)
    dirv /= np.linalg.norm(dirv)
    xt = cen + dist * L * dirv
    nt = rng.standard_normal(3)
    nt /= np.linalg.norm(nt)
    tg = W.Targets(xt[None], nt[None], np.array([-1]))
    v128, _, flags = o128.rows(tg, [0], [0])
    assert flags[0] == 0
    uv = W.ref_nodes(p)
    sig = _mu(uv[:, 0], uv[:, 1])
    with mp.workdps(30):
        for k in KINDS:
            sm = sum(brute.kernel(k, xt, nt, d.xyz[i][None], d.nrm[i][None])[0] * d.wts[i] * sig[i]
                     for i in range(len(sig)))
            # the RRQ part in binary64: (correction + smooth), each rounded once
            got = mp.fsum([mp.mpf(float(v)) * mp.mpf(float(s)) for v, s in zip(v128[k], sig)]) + mp.mpf(float(sm))
            ex = _exact(k, xt, nt)
            # rounding of the binary64 outputs: |row| |sig| 2^-53 per entry, and of sm
            eout = (np.abs(v128[k]) @ np.abs(sig) + abs(sm)) * 2.0 ** -52
            assert abs(got - ex) <= max(2e-15 * abs(ex), eout), (k, float(got), float(ex))


def test_f128_agrees_with_binary64(O):
    """Same algorithm: on the unit sphere at p = 4 (well conditioned) the two builds agree
    to binary64 rounding, row by row."""
    d, tg = W.sphere80(4)
    sel = np.arange(0, tg.n, 11)
    rp, col, v64, _ = O.OracleSurface(d).csr_rows(tg, sel)
    rp2, col2, v128, _ = O.OracleSurface(d, ext=True).csr_rows(tg, sel)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    for k in KINDS:
        scale = np.maximum(np.abs(v128[k]), 1.0)
        assert np.max(np.abs(v64[k] - v128[k]) / scale) < 1e-12, k
