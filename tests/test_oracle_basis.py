"""Pins of the oracle's harmonic polynomials and 1-D quadrature pieces.

Each check compares against mathematics that does not come from the oracle's own
formulas: the addition theorem evaluated at independent points, the spherical
harmonic addition identity, finite differences, Laplace's equation, the flat
triangle theorem, textbook moments and scipy adaptive quadrature.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from paper_2411_08342_gb300 import workloads as W


def test_addition_theorem(oracle_lib):
    """R_l^m(a+b) = sum_{j,k} R_j^k(a) R_{l-j}^{m-k}(b) T_{jk,lm} (Sec. 2.3, eqs.
    l2ltranslation, tjklmdef) for random a, b: pins the Legendre recurrence, the
    normalisation of R_l^m and the negative-m convention together."""
    O = oracle_lib
    rng = np.random.default_rng(7)
    L = 10
    for _ in range(3):
        a = rng.standard_normal(3) * 0.6
        b = rng.standard_normal(3) * 0.6
        Ra, Rb, Rab = O.solid_R(L, a), O.solid_R(L, b), O.solid_R(L, a + b)
        for l in range(L + 1):
            for m in range(-l, l + 1):
                s = 0
                for j in range(l + 1):
                    for k in range(-j, j + 1):
                        if abs(m - k) > l - j:
                            continue
                        s += Ra[O.hidx(j, k)] * Rb[O.hidx(l - j, m - k)] * O.T(j, k, l, m)
                assert abs(s - Rab[O.hidx(l, m)]) < 1e-13 * (1 + abs(Rab[O.hidx(l, m)]))


def test_spherical_addition_identity(oracle_lib):
    """sum_m |Y_l^m|^2 = 2l+1 with the paper's normalisation (no 1/sqrt(4 pi)),
    i.e. sum_m |R_l^m(x)|^2 = |x|^{2l}."""
    O = oracle_lib
    rng = np.random.default_rng(2)
    x = rng.standard_normal(3)
    R = O.solid_R(9, x)
    r2 = x @ x
    for l in range(10):
        s = sum(abs(R[O.hidx(l, m)]) ** 2 for m in range(-l, l + 1))
        assert abs(s - r2 ** l) < 1e-13 * r2 ** l


def test_low_degree_closed_forms(oracle_lib):
    """R_0^0 = 1, R_1^0 = z, |R_1^1| = rho/sqrt2, R_2^0 = (2z^2 - x^2 - y^2)/2."""
    O = oracle_lib
    x = np.array([0.3, -0.7, 0.45])
    R = O.solid_R(2, x)
    assert abs(R[O.hidx(0, 0)] - 1) < 1e-15
    assert abs(R[O.hidx(1, 0)] - x[2]) < 1e-15
    assert abs(abs(R[O.hidx(1, 1)]) - math.hypot(x[0], x[1]) / math.sqrt(2)) < 1e-15
    assert abs(R[O.hidx(2, 0)] - (2 * x[2] ** 2 - x[0] ** 2 - x[1] ** 2) / 2) < 1e-15
    # S(x,y,z) = R(y,z,x): the polar axis of S is the x axis
    S = O.solid_S(2, x)
    assert abs(S[O.hidx(1, 0)] - x[0]) < 1e-15


@pytest.mark.parametrize("lm", [(2, 1), (4, -3), (7, 7), (8, 0), (6, 2)])
def test_gradient_hessian_finite_difference(oracle_lib, lm):
    O = oracle_lib
    l, m = lm
    y = np.array([0.21, -0.33, 0.17])
    g, H = O.grad_hess_S(8, y, l, m)
    h = 1e-4
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (-O.solid_S(8, y + 2 * e) + 8 * O.solid_S(8, y + e) - 8 * O.solid_S(8, y - e)
              + O.solid_S(8, y - 2 * e)) / (12 * h)
        assert abs(fd[O.hidx(l, m)] - g[a]) < 1e-10
        g1, _ = O.grad_hess_S(8, y + e, l, m)
        g2, _ = O.grad_hess_S(8, y - e, l, m)
        assert np.abs((g1 - g2) / (2 * h) - H[:, a]).max() < 1e-7
    # harmonic: Laplacian from second differences of the values
    lap = 0
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1e-3
        lap += (O.solid_S(8, y + e) - 2 * O.solid_S(8, y) + O.solid_S(8, y - e))[O.hidx(l, m)] / 1e-6
    assert abs(lap) < 1e-5


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_flat_triangle_basis_theorem(oracle_lib, p):
    """Thm. trianglebasis: on z = 0, H^{(l,m)} = sqrt2 Im S^{(l,m)} vanishes, grad H is
    along e_z, and F^{(l,m)} = dH/dz span all polynomials of degree <= p-1."""
    O = oracle_lib
    rng = np.random.default_rng(p)
    pts = rng.random((3 * p * p, 2)) - 0.5
    F = []
    for (x, y) in pts:
        S = O.solid_S(p, [x, y, 0.0])
        row = []
        for l in range(1, p + 1):
            for m in range(1, l + 1):
                assert abs(math.sqrt(2) * S[O.hidx(l, m)].imag) < 1e-15
                g, _ = O.grad_hess_S(p, [x, y, 0.0], l, m)
                Hg = math.sqrt(2) * g.imag
                assert abs(Hg[0]) < 1e-14 and abs(Hg[1]) < 1e-14
                row.append(Hg[2])
        F.append(row)
    F = np.array(F)
    mono = np.array([[x ** a * y ** b for a in range(p) for b in range(p - a)] for (x, y) in pts])
    # span equality: ranks of F, mono and [F mono] are all n_p
    npn = p * (p + 1) // 2
    assert np.linalg.matrix_rank(F, tol=1e-10) == npn
    assert np.linalg.matrix_rank(np.hstack([F, mono]), tol=1e-9) == npn


def test_gauss_legendre_exactness(oracle_lib):
    O = oracle_lib
    for n in (4, 8, 16, 32):
        x, w = O.gauss_legendre(n)
        for k in range(2 * n):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("ab", [(0.3, 0.05), (-0.9, 1e-4), (1.2, 0.02), (0.0, 0.7), (0.5, 1e-7)])
def test_ssq_moments_against_adaptive_quadrature(oracle_lib, ab):
    """I_i = int t^i / ((t-a)^2+b^2)^{m/2} dt (Sec. 2.4, eq. ssq1dintegrals) for m = 1, 3."""
    O = oracle_lib
    a, b = ab
    J, K = O.ssq_moments(16, a, b)
    # reference by the substitution t - a = b sinh(s), which removes the near singularity
    lo, hi = math.asinh((-1 - a) / b), math.asinh((1 - a) / b)
    for i in range(16):
        rj = quad(lambda s: (a + b * math.sinh(s)) ** i, lo, hi, limit=500, epsabs=0, epsrel=1e-13)[0]
        rk = quad(lambda s: (a + b * math.sinh(s)) ** i / (b * math.cosh(s)) ** 2, lo, hi, limit=500,
                  epsabs=0, epsrel=1e-13)[0]
        assert abs(J[i] - rj) < 1e-12 * max(1.0, abs(J[0]))
        assert abs(K[i] - rk) < 1e-11 * max(1.0, abs(K[0]))


@pytest.mark.parametrize("ab", [(0.3, 0.05), (-0.9, 1e-4), (1.2, 0.02), (0.0, 0.7), (0.5, 1e-7)])
def test_ssq_weights_high_order(oracle_lib, ab):
    """The edge rule's singularity-swap weights lambda (V^T lambda = I, Sec. 3.4) integrate
    f(t) / ((t-a)^2+b^2)^{m/2} for a smooth f to near machine precision up to pt = 28
    nodes (order p = 14), although cond(V) reaches 1e10 there: the system is solved by a
    backward stable method (Sec. 5.1).  A rule formed as U^T I with the explicit inverse U
    loses ~8 digits at pt = 24 to cancellation.  Reference by the sinh substitution."""
    O = oracle_lib
    a, b = ab
    f = lambda t: np.exp(t) * np.cos(2 * t)
    lo, hi = math.asinh((-1 - a) / b), math.asinh((1 - a) / b)
    r1 = quad(lambda s: f(a + b * math.sinh(s)), lo, hi, limit=500, epsabs=0, epsrel=1e-13)[0]
    r3 = quad(lambda s: f(a + b * math.sinh(s)) / (b * math.cosh(s)) ** 2, lo, hi, limit=500, epsabs=0,
              epsrel=1e-13)[0]
    for pt in (20, 24, 28):
        x, _ = O.gauss_legendre(pt)
        l1, l3 = O.ssq_weights(pt, a, b)
        assert abs(l1 @ f(x) - r1) <= 2e-13 * abs(r1), (pt, l1 @ f(x), r1)
        assert abs(l3 @ f(x) - r3) <= 2e-13 * abs(r3), (pt, l3 @ f(x), r3)


def test_bernstein_radius(oracle_lib):
    O = oracle_lib
    assert abs(O.bernstein_rho(0.3 + 0j) - 1.0) < 1e-14
    assert abs(O.bernstein_rho(2.0 + 0j) - (2 + math.sqrt(3))) < 1e-13
    assert abs(O.bernstein_rho(1j) - (1 + math.sqrt(2))) < 1e-13


def test_lu_solve(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40))
    B = rng.standard_normal((40, 3))
    assert np.abs(O.lu_solve(A, B) - np.linalg.solve(A, B)).max() < 1e-12


def test_fit_condition_number(oracle_lib):
    """kappa_1 of the fit matrix A of eq. dlpdensitylinearsystem2 (the oracle's, from its LU
    inverse) equals numpy's 1-norm condition number of the same block matrix built here
    from the harmonic gradients at the patch's local nodes, and grows with curvature and
    order (Sec. 5.1)."""
    O = oracle_lib
    ks = {}
    for p, lev in ((4, 1), (6, 1), (6, 3)):
        d = W.discretize(W.star_surface(lev), p)
        osf = O.OracleSurface(d)
        info = osf.patch_internals(0)
        y = info["y"]
        npn = p * (p + 1) // 2
        _, gH = O.basis_batch(p, y)
        A = np.zeros((4 * npn, 4 * npn))
        for i in range(npn):
            for lm in range(npn):
                f1, f2, f3 = gH[i, lm]
                blk = [[0, -f1, -f2, -f3], [f1, 0, -f3, f2], [f2, f3, 0, -f1], [f3, -f2, f1, 0]]
                for r in range(4):
                    for c in range(4):
                        A[r * npn + i, c * npn + lm] = blk[r][c]
        k_np = np.linalg.cond(A, 1)
        k_or = osf.patch_kappa(0)
        assert abs(k_or - k_np) <= 1e-8 * k_np, (p, lev, k_or, k_np)
        ks[(p, lev)] = k_or
    assert ks[(6, 1)] > ks[(4, 1)]          # higher order on the same patch
    assert ks[(6, 1)] > ks[(6, 3)]          # coarser (more curved) patch at the same order


def _paraboloid_kappa(O, H, h, p, R=None, shift=None):
    d = W.discretize(W.paraboloid_patch(H, h), p)
    if R is not None:
        d.xyz = d.xyz @ R.T + shift
        d.nrm = d.nrm @ R.T
    return O.OracleSurface(d).patch_kappa(0)


def test_fit_condition_paraboloid(oracle_lib):
    """kappa_1(A) on the paraboloid patch of eq. (paraboloid), against what Step 1 and
    Sec. 5.1 fix:
      * Step 1 scales the patch to unit longest side, so a patch of side h and curvature H
        has the kappa of side 1 and curvature H h (exactly, up to rounding);
      * Step 1 also removes rigid motions: a rotated and shifted patch has the same kappa;
      * a small patch is nearly flat, so kappa(H, h) tends to the flat triangle's value as
        h -> 0 (the right panel of the conditioning figure), decreasing on the way;
      * on the flat triangle kappa grows with p (the left panel of the second figure)."""
    O = oracle_lib
    rot = np.array([[0.36, -0.48, 0.8], [0.8, 0.6, 0.0], [-0.48, 0.64, 0.6]])  # orthogonal
    assert np.abs(rot @ rot.T - np.eye(3)).max() < 1e-15
    flat = [_paraboloid_kappa(O, 0.0, 1.0, p) for p in range(2, 9)]
    assert all(b > 3.0 * a for a, b in zip(flat, flat[1:])), flat
    for p in (4, 6, 8):
        k = _paraboloid_kappa(O, 10.0, 0.3, p)
        assert abs(k / _paraboloid_kappa(O, 3.0, 1.0, p) - 1) < 1e-9, p
        k_rot = _paraboloid_kappa(O, 3.0, 1.0, p, rot, np.array([1.0, -2.0, 0.5]))
        assert abs(k_rot / _paraboloid_kappa(O, 3.0, 1.0, p) - 1) < 1e-9, p
        seq = [_paraboloid_kappa(O, 10.0, 2.0 ** -L, p) for L in (2, 4, 6, 8, 10)]
        assert all(b < a for a, b in zip(seq, seq[1:])), (p, seq)
        assert abs(seq[-1] / flat[p - 2] - 1) < 0.03, (p, seq[-1], flat[p - 2])
        assert _paraboloid_kappa(O, 10.0, 1.0, p) > 10 * flat[p - 2]


def test_quaternion_interpolation_converges(oracle_lib):
    """The quaternion harmonic fit of Sec. 3.2 (eq. dlpdensitylinearsystem2) on a flat
    equilateral triangle of side 1 centred at the origin, as in the interpolation study of
    Sec. 5.1: the scalar part of q = sum_lm (0, grad H^{(l,m)}) c^{(l,m)} reproduces the
    density at the nodes (collocation) and, for the analytic densities of that study,
    converges geometrically in p away from the nodes."""
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
    funcs = {"1/(x^2+y^2+0.5)": lambda x, y: 1 / (x * x + y * y + 0.5),
             "cos(12x+12y+1)": lambda x, y: np.cos(12 * x + 12 * y + 1)}
    err = {}
    for p in (4, 6, 8, 10, 12):
        d = W.discretize(W.flat_surface(tri), p)
        info = O.OracleSurface(d).patch_internals(0)
        npn = p * (p + 1) // 2
        fr = info["frame"]
        c0, Rm, s = fr[:3], fr[3:12].reshape(3, 3), fr[12]
        XD = info["XD"].reshape(4, npn, npn)
        for name, f in funcs.items():
            mu = f(d.xyz[:, 0], d.xyz[:, 1])
            c = np.einsum("qli,i->lq", XD, mu)
            def q0(P):
                _, gH = O.basis_batch(p, s * (P - c0) @ Rm)
                return -np.einsum("mla,la->m", gH, c[:, 1:])
            assert np.abs(q0(d.xyz) - mu).max() < 1e-9 * np.abs(mu).max(), (p, name)
            ref = f(pts[:, 0], pts[:, 1])
            err[(name, p)] = np.abs(q0(pts) - ref).max() / np.abs(ref).max()
    e1 = [err[("1/(x^2+y^2+0.5)", p)] for p in (4, 6, 8, 10, 12)]
    assert all(b_ < a_ / 3 for a_, b_ in zip(e1, e1[1:])), e1
    assert e1[-1] < 1e-5, e1
    e2 = [err[("cos(12x+12y+1)", p)] for p in (4, 6, 8, 10, 12)]
    assert e2[-1] < e2[0] / 20, e2


def test_reference_rule_moments():
    """The smooth rule of the synthetic inputs (workloads.ref_weights at workloads.ref_nodes)
    integrates every monomial u^a v^b of total degree < p exactly over the reference
    triangle (a! b! / (a + b + 2)!), to rounding, for every order up to 12; the nodes lie
    strictly inside the triangle."""
    for p in range(2, 13):
        uv = W.ref_nodes(p)
        w = W.ref_weights(p)
        assert len(uv) == p * (p + 1) // 2
        assert np.all(uv > 0) and np.all(uv.sum(1) < 1)
        for a in range(p):
            for b in range(p - a):
                exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                assert abs(np.sum(w * uv[:, 0] ** a * uv[:, 1] ** b) - exact) < 1e-15, (p, a, b)
