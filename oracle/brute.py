"""Brute-force surface quadrature used to pin the oracle (test infrastructure).

Nothing here shares arithmetic with rrq_oracle.c: the layer potentials are
integrated directly from their definitions (Sec. 1, eqs. slpdef-dprimelpdef,
G = 1/(4 pi |r'-r|)) with adaptive / graded Gauss rules.

* ``flat_triangle``: a planar triangle and a density that is a polynomial of the
  reference coordinates.  The triangle is split into three signed triangles at the
  foot point of the target; each is integrated in polar coordinates (radius graded
  geometrically toward the target height, angle by adaptive Gauss-Kronrod).
* ``curved_patch``: a curved patch X(u,v) and a smooth integrand, integrated by
  recursive 4-way subdivision of the reference triangle until every piece is far
  from the target relative to its size, with a collapsed Gauss rule per piece.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad

INV4PI = 1.0 / (4.0 * np.pi)


def kernel(kind: str, tgt, tnrm, r, nrm):
    """K(r', r) for kind in S, D, SP, DP at source points r (..., 3) with normals nrm."""
    return kernel_d(kind, tgt - r, tnrm, nrm)


def kernel_d(kind: str, d, tnrm, nrm):
    """The same kernels as functions of d = r' - r."""
    r2 = np.einsum("...a,...a->...", d, d)
    rr = np.sqrt(r2)
    if kind == "S":
        return INV4PI / rr
    if kind == "D":
        return INV4PI * np.einsum("...a,...a->...", d, nrm) / (r2 * rr)
    if kind == "SP":
        return -INV4PI * np.einsum("...a,...a->...", d, tnrm) / (r2 * rr)
    if kind == "DP":
        dn = np.einsum("...a,...a->...", d, nrm)
        dt = np.einsum("...a,...a->...", d, tnrm)
        return INV4PI * (np.einsum("...a,...a->...", nrm * np.ones_like(d), tnrm * np.ones_like(d)) / (r2 * rr)
                         - 3.0 * dn * dt / (r2 * r2 * rr))
    raise ValueError(kind)


def _radial_panels(h: float, R: float, n: int = 20):
    """Graded Gauss nodes on [0, R] toward 0 at scale max(h, tiny)."""
    x, w = np.polynomial.legendre.leggauss(n)
    s = max(h, 1e-14 * max(R, 1e-300))
    br = [0.0]
    t = s / 2
    while t < R:
        br.append(t)
        t *= 2.0
    br.append(R)
    br = np.array(br)
    a, b = br[:-1], br[1:]
    nodes = (0.5 * (a + b))[:, None] + (0.5 * (b - a))[:, None] * x[None, :]
    wts = (0.5 * (b - a))[:, None] * w[None, :]
    return nodes.ravel(), wts.ravel()


def flat_triangle(kind: str, A, B, C, tgt, tnrm, mu, epsrel: float = 1e-13):
    """int over triangle ABC of K(tgt, r) mu(u, v) da, normal = unit((B-A) x (C-A)),
    mu a callable of reference coordinates (u, v) (r = A + u (B-A) + v (C-A))."""
    A, B, C, tgt, tnrm = (np.asarray(v, dtype=np.float64) for v in (A, B, C, tgt, tnrm))
    n = np.cross(B - A, C - A)
    area2 = np.linalg.norm(n)
    nu = n / area2
    h = float(np.dot(tgt - A, nu))
    p0 = tgt - h * nu
    e1 = (B - A) / np.linalg.norm(B - A)
    e2 = np.cross(nu, e1)
    # reference coordinates of a plane point: solve r - A = u (B-A) + v (C-A)
    M = np.stack([B - A, C - A], 1)
    Mp = np.linalg.pinv(M)

    def integrate_sub(P1, P2):
        # signed triangle (p0, P1, P2)
        q1, q2 = P1 - p0, P2 - p0
        a1 = np.arctan2(np.dot(q1, e2), np.dot(q1, e1))
        a2 = np.arctan2(np.dot(q2, e2), np.dot(q2, e1))
        da = a2 - a1
        while da > np.pi:
            da -= 2 * np.pi
        while da < -np.pi:
            da += 2 * np.pi
        if abs(da) < 1e-15:
            return 0.0
        edge = P2 - P1
        nrm_e = np.cross(nu, edge)     # in-plane normal of the line P1P2
        dist = np.dot(P1 - p0, nrm_e) / np.linalg.norm(nrm_e)

        def f_theta(th):
            dirv = np.cos(th) * e1 + np.sin(th) * e2
            den = np.dot(dirv, nrm_e) / np.linalg.norm(nrm_e)
            if abs(den) < 1e-300:
                return 0.0
            R = dist / den
            if R <= 0:
                return 0.0
            rho, w = _radial_panels(abs(h), R)
            pts = p0[None, :] + rho[:, None] * dirv[None, :]
            uv = (pts - A[None, :]) @ Mp.T
            dvec = h * nu[None, :] - rho[:, None] * dirv[None, :]   # r' - r without cancellation
            k = kernel_d(kind, dvec, tnrm, nu[None, :])
            return float(np.sum(w * rho * k * mu(uv[:, 0], uv[:, 1])))

        # the line P1P2 is closest to p0 at angle th_n: split there for smoothness
        th_n = np.arctan2(np.dot(nrm_e, e2), np.dot(nrm_e, e1))
        lo, hi = (a1, a1 + da) if da > 0 else (a1 + da, a1)
        pts = []
        for k in (-2, -1, 0, 1, 2):
            t = th_n + 2 * np.pi * k
            if lo < t < hi:
                pts.append(t)
        val, _ = quad(f_theta, lo, hi, points=pts or None, limit=400, epsabs=0.0, epsrel=epsrel)
        return val if da > 0 else -val

    return integrate_sub(A, B) + integrate_sub(B, C) + integrate_sub(C, A)


def _tri_rule(n: int):
    """Collapsed (Duffy) Gauss rule on the reference triangle with n x n points."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = (x + 1) / 2
    w = w / 2
    U, V = np.meshgrid(x, x, indexing="ij")
    Wt = np.outer(w, w)
    u = U * (1 - V)
    v = V
    return np.stack([u.ravel(), v.ravel()], 1), (Wt * (1 - V)).ravel()


def curved_patch(integrand, X, tgt, size_ratio: float = 3.0, n: int = 14, max_depth: int = 14):
    """int over T of integrand(uv, X(uv), Xu x Xv) du dv by recursive subdivision.
    The integrand may return (m,) or (m, ...) values for the m points.

    X(uv) -> (points (m,3), cross (m,3)) where cross = X_u x X_v (area element and
    normal).  A piece is accepted when its diameter * size_ratio < distance to tgt."""
    uvq, wq = _tri_rule(n)
    tgt = np.asarray(tgt, dtype=np.float64)
    total = 0.0
    stack = [(np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0]), 0)]
    while stack:
        a, b, c, dep = stack.pop()
        corners = np.stack([a, b, c, (a + b + c) / 3])
        pc, _ = X(corners)
        diam = max(np.linalg.norm(pc[0] - pc[1]), np.linalg.norm(pc[1] - pc[2]), np.linalg.norm(pc[2] - pc[0]))
        dist = np.min(np.linalg.norm(pc - tgt[None, :], axis=1)) - diam
        if dep < max_depth and dist < size_ratio * diam:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            stack += [(a, ab, ca, dep + 1), (ab, b, bc, dep + 1), (ca, bc, c, dep + 1), (ab, bc, ca, dep + 1)]
            continue
        jac = abs((b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]))
        uv = a[None, :] + uvq[:, 0:1] * (b - a)[None, :] + uvq[:, 1:2] * (c - a)[None, :]
        pts, cr = X(uv)
        vals = np.asarray(integrand(uv, pts, cr))
        total = total + jac * np.tensordot(wq, vals, axes=(0, 0))
    return total
