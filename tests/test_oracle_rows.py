"""Pins of the oracle's correction rows against brute force and closed forms.

* flat triangles: for a density that is a polynomial of degree <= p-1 the quaternion
  and scalar fits are exact on a flat patch (Thm. trianglebasis and the remarks after
  eq. dlpdensitylinearsystem2), so RRQ row . mu must equal the layer potential of mu
  computed by brute force from the definitions (eqs. slpdef-dprimelpdef);
* Omega_0 against the Van Oosterom-Strackee solid angle of a flat triangle;
* curved patches: the line-integral quantities B^{(l,m)} and Psi^{(l,m)} against
  brute-force surface integrals of the 2-forms alpha^{(l,m)} (eq. dlp2form) and
  chi^{(l,m)} (eq. slp2form);
* closed surfaces: Gauss's law for D[1] and the spherical-harmonic eigenvalues of
  S, D, S', D' on the unit sphere (whole operator = smooth rule + correction).
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


def rrq_value(d, vals, kind, sig, xt, nt, self_i=-1):
    """RRQ part of a single-pair row: correction + smooth (and jump removed)."""
    r = vals[kind] @ sig
    for i in range(len(sig)):
        if i == self_i:
            continue
        r += brute.kernel(kind, xt, nt, d.xyz[i][None], d.nrm[i][None])[0] * d.wts[i] * sig[i]
    return r


@pytest.fixture(scope="module")
def flat5(oracle_lib):
    d = W.discretize(W.flat_surface(np.array([[A, B, C]])), 5)
    return d, oracle_lib.OracleSurface(d)


FLAT_TARGETS = [
    ("above", (A + B + C) / 3 + 0.1 * E1 + 0.05 * NU),
    ("close", (A + B + C) / 3 + 0.1 * E1 + 1e-4 * NU),
    ("below", (A + B + C) / 3 - 0.1 * E2 - 0.02 * NU),
    ("edge_out", (A + B) / 2 - 1e-3 * E2 + 1e-4 * NU),
    ("edge_in", (A + B) / 2 + 0.05 * E2 + 0.01 * NU),
    ("far", A + 0.3 * (B - A) + 0.2 * NU),
]


@pytest.mark.parametrize("name,xt", FLAT_TARGETS, ids=[t[0] for t in FLAT_TARGETS])
def test_flat_triangle_rows_equal_brute_force(flat5, name, xt):
    d, osf = flat5
    rng = np.random.default_rng(abs(hash(name)) % 1000)
    nt = rng.standard_normal(3)
    nt /= np.linalg.norm(nt)
    tg = W.Targets(xt[None], nt[None], np.array([-1]))
    vals, _, flags = osf.rows(tg, [0], [0])
    assert flags[0] == 0
    uv = W.ref_nodes(5)
    sig = _mu(uv[:, 0], uv[:, 1])
    for kind in KINDS:
        got = rrq_value(d, vals, kind, sig, xt, nt)
        ref = brute.flat_triangle(kind, A, B, C, xt, nt, _mu)
        assert abs(got - ref) < 2e-11 * max(1.0, abs(ref)), (kind, got, ref)


def test_flat_triangle_self_rows(flat5):
    """On-surface nodes of a flat patch: D_pv[mu] = 0 and S'_pv = 0 on a plane; S
    equals the weakly singular integral computed by polar brute force."""
    d, osf = flat5
    uv = W.ref_nodes(5)
    sig = _mu(uv[:, 0], uv[:, 1])
    for i in (0, 7, 14):
        tg = W.Targets(d.xyz[i][None], d.nrm[i][None], np.array([i]))
        vals, _, _ = osf.rows(tg, [0], [0], ("S", "D", "SP"))
        xt = d.xyz[i]
        s = rrq_value(d, vals, "S", sig, xt, d.nrm[i], i)
        assert abs(s - brute.flat_triangle("S", A, B, C, xt, NU, _mu)) < 1e-11
        assert abs(rrq_value(d, vals, "D", sig, xt, d.nrm[i], i)) < 1e-12
        assert abs(rrq_value(d, vals, "SP", sig, xt, d.nrm[i], i)) < 1e-12


def _vos(xt, P0, P1, P2):
    R1, R2, R3 = P0 - xt, P1 - xt, P2 - xt
    r1, r2, r3 = (np.linalg.norm(v) for v in (R1, R2, R3))
    return 2 * math.atan2(R1 @ np.cross(R2, R3),
                          r1 * r2 * r3 + (R1 @ R2) * r3 + (R1 @ R3) * r2 + (R2 @ R3) * r1)


def test_solid_angle_van_oosterom_strackee(flat5):
    """Omega_0 / (4 pi) = -int grad_r G . nu da = VOS(r') / (4 pi) for a flat triangle
    (with this vertex order the Van Oosterom-Strackee formula is signed the same way)."""
    d, osf = flat5
    info = osf.patch_internals(0)
    for name, xt in FLAT_TARGETS + [("vertex_near", A + 1e-3 * (B + C - 2 * A) + 1e-6 * NU)]:
        r = osf.pair_B(0, xt, NU)
        assert abs(r["Om"][0] - _vos(xt, A, B, C)) < 1e-12, name
    assert info["status"] == 0


def _patch_map(d, P, info):
    """Local-frame map y(u,v) of patch P from its node interpolant, with y_u x y_v."""
    p = int(d.order[P])
    uvn = d.ref_uv[p]
    xn = d.xyz[d.node_off[P]:d.node_off[P + 1]]
    c, R, s = info["c"], info["R"], info["s"]
    yn = s * (xn - c) @ R

    def X(uv):
        uvc = uv.astype(np.complex128)
        M = W.interp_matrix(uvn, p, uv)
        pts = M @ yn
        h = 1e-30
        Mu = W.interp_matrix(uvn, p, uvc + np.array([1j * h, 0]))
        Mv = W.interp_matrix(uvn, p, uvc + np.array([0, 1j * h]))
        yu = (Mu @ yn).imag / h
        yv = (Mv @ yn).imag / h
        return pts, np.cross(yu, yv)
    return X


def _qmul(f, g):
    """Quaternion product of arrays (..., 4) (eq. qprule)."""
    f0, fv, g0, gv = f[..., 0], f[..., 1:], g[..., 0], g[..., 1:]
    s = f0 * g0 - np.einsum("...a,...a->...", fv, gv)
    v = f0[..., None] * gv + g0[..., None] * fv + np.cross(fv, gv)
    return np.concatenate([s[..., None], v], -1)


@pytest.mark.parametrize("case", ["off_center", "near_edge", "beyond_edge"])
def test_curved_patch_stokes_reduction(oracle_lib, case):
    """B^{(l,m)} = int_P alpha^{(l,m)} and Psi^{(l,m)} = int_P chi^{(l,m)} on a curved
    patch of the unit sphere (Thms. dlp1form, cslp1form; eqs. dlp2form, slp2form),
    the surface integrals done by brute force in the patch's local frame.  The edge
    rule is refined to ptilde = 12 nodes so that the line quadrature resolves these
    strongly curved edges (with ptilde = 2p = 8 the check holds to ~1e-7; beyond
    ptilde ~ 14 the monomial Vandermonde of Sec. 3.4 loses digits)."""
    O = oracle_lib
    p = 4
    d = W.discretize(W.sphere_surface(1), p)
    osf = O.OracleSurface(d, ptilde=12)
    P = 3
    info = osf.patch_internals(P)
    c, R, s = info["c"], info["R"], info["s"]
    X = _patch_map(d, P, info)
    if case == "off_center":
        yt = np.array([0.05, 0.02, 0.15])
    elif case == "near_edge":
        e = info["ey"][0]
        yt = e[len(e) // 2] + np.array([0.0, 0.01, 0.02])
    else:
        e = info["ey"][1]
        mid = e[len(e) // 2]
        yt = mid + 0.03 * mid / np.linalg.norm(mid) + np.array([0, 0, 0.01])
    xt = c + (R @ yt) / s
    nt = R @ np.array([0.3, -0.2, 0.93])
    nt /= np.linalg.norm(nt)
    r = osf.pair_B(P, xt, nt)

    npn = p * (p + 1) // 2

    def integrand(uv, pts, cr):
        dv = yt[None, :] - pts
        rr = np.linalg.norm(dv, axis=1)
        G = 1 / (4 * np.pi * rr)
        gG = dv / (4 * np.pi * rr[:, None] ** 3)              # grad_r G
        H, gH = O.basis_batch(p, pts)                          # (m, npn), (m, npn, 3)
        z = np.zeros((len(pts), 1))
        q12 = _qmul(np.concatenate([z, gG], 1), np.concatenate([z, cr], 1))      # (0,grad G)(0, nu da)
        q3 = np.concatenate([np.zeros(gH.shape[:2] + (1,)), gH], 2)
        alpha = _qmul(np.broadcast_to(q12[:, None, :], q3.shape), q3)            # (m, npn, 4)
        chi = np.einsum("ija,ia->ij", G[:, None, None] * gH - H[:, :, None] * gG[:, None, :], cr)
        return np.concatenate([alpha.reshape(len(pts), -1), chi], 1)

    ref = brute.curved_patch(integrand, X, yt, n=12, size_ratio=2.0)
    ref_alpha = ref[:4 * npn].reshape(npn, 4)
    ref_chi = ref[4 * npn:]
    scale = np.abs(ref_alpha).max()
    assert np.abs(r["B"] - ref_alpha).max() < 2e-11 * scale
    assert np.abs(r["Psi"] - ref_chi).max() < 2e-11 * np.abs(ref_chi).max()
    # d B / d nu' against a central difference of the line-integral B in the nu' direction
    h = 2e-4
    nl = R.T @ nt
    Bs = {k: osf.pair_B(P, c + (R @ (yt + k * h * nl)) / s, nt)["B"] for k in (-2, -1, 1, 2)}
    fd = (Bs[-2] - 8 * Bs[-1] + 8 * Bs[1] - Bs[2]) / (12 * h)
    assert np.abs(r["dB"] - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def _apply_whole(d, tg, rowptr, col, val, kind, sig):
    out = np.zeros(tg.n)
    for c0 in range(0, tg.n, 1024):
        t = tg.xyz[c0:c0 + 1024]
        tn = tg.nrm[c0:c0 + 1024]
        with np.errstate(divide="ignore", invalid="ignore"):
            K = brute.kernel(kind, t[:, None, :], tn[:, None, :], d.xyz[None], d.nrm[None])
        sn = tg.self_node[c0:c0 + 1024]
        K[np.arange(len(t))[sn >= 0], sn[sn >= 0]] = 0
        out[c0:c0 + 1024] = K @ (d.wts * sig)
    return out + np.add.reduceat(val * sig[col], rowptr[:-1])


def test_sphere_eigenvalues_converge(oracle_lib):
    """On the unit sphere: S[Y_l] = Y_l/(2l+1), D_pv[Y_l] = S'_pv[Y_l] = -Y_l/(2(2l+1)),
    D'[Y_l] = -l(l+1)/(2l+1) Y_l.  The full operator (smooth rule + correction) must
    approach these at high order as the mesh is refined (p = 4: 80 -> 320 patches)."""
    O = oracle_lib
    l, m = 2, 1
    ev = {"S": 1 / (2 * l + 1), "D": -1 / (2 * (2 * l + 1)), "SP": -1 / (2 * (2 * l + 1)),
          "DP": -l * (l + 1) / (2 * l + 1)}
    errs = {}
    for lev in (1, 2):
        d = W.discretize(W.sphere_surface(lev), 4)
        tg = W.on_surface_targets(d)
        osf = O.OracleSurface(d)
        rowptr, col, vals, flags = osf.csr_rows(tg)
        Y = W.real_ylm(l, m, d.xyz)
        for k in KINDS:
            y = _apply_whole(d, tg, rowptr, col, vals[k], k, Y)
            errs[(lev, k)] = np.abs(y - ev[k] * Y).max() / np.abs(ev[k] * Y).max()
    for k in KINDS:
        assert errs[(2, k)] < 1e-2, errs
        assert errs[(1, k)] / errs[(2, k)] > 6.0, errs     # better than O(h^2.5) per halving
    assert errs[(2, "S")] < 5e-4


def test_gauss_law(oracle_lib):
    """D[1] = -1 inside, -1/2 on the surface (principal value), 0 outside, for a closed
    star-shaped surface.  Neighbouring patch interpolants meet only to O(h^p) along
    shared edges (interior nodes), so the check is convergence: 320 -> 1280 patches."""
    O = oracle_lib
    errs = []
    for lev in (2, 3):
        d = W.discretize(W.star_surface(lev, terms=((2, 1, 0.15), (3, 2, 0.1))), 5)
        rng = np.random.default_rng(5)
        on = W.on_surface_targets(d)
        sel = rng.choice(on.n, 40, replace=False)
        idx = rng.integers(0, d.nnode, 40)
        xin = d.xyz[idx] - 0.01 * d.nrm[idx]
        xout = d.xyz[idx] + 0.01 * d.nrm[idx]
        tg = W.concat_targets(W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel]),
                              W.Targets(xin, d.nrm[idx], -np.ones(40, np.int64)),
                              W.Targets(xout, d.nrm[idx], -np.ones(40, np.int64)))
        osf = O.OracleSurface(d)
        rowptr, col, vals, _ = osf.csr_rows(tg, kernels=("D",))
        y = _apply_whole(d, tg, rowptr, col, vals["D"], "D", np.ones(d.nnode))
        errs.append(max(np.abs(y[:40] + 0.5).max(), np.abs(y[40:80] + 1.0).max(), np.abs(y[80:]).max()))
    assert errs[1] < 5e-5, errs
    assert errs[0] / errs[1] > 5.0, errs


def test_edge_root(oracle_lib):
    """t0 solves sum_a (y_a(t0) - y'_a)^2 = 0 (eq. complexparameter) with Im t0 > 0 and
    is the root nearest the chord estimate among the polynomial's roots."""
    O = oracle_lib
    d = W.discretize(W.sphere_surface(1), 6)
    osf = O.OracleSurface(d)
    info = osf.patch_internals(5)
    p = 6
    for e in range(3):
        mid = info["ey"][e][6]
        yt = mid + np.array([0.01, -0.02, 0.03])
        t0, conv = osf.edge_root(5, e, yt)
        assert conv and t0.imag > 0
        # polynomial in t via the Legendre coefficients
        coef = info["ea"][e]                       # (p, 3)
        poly = [np.polynomial.legendre.leg2poly(coef[:, a]) for a in range(3)]
        g = sum(np.polynomial.polynomial.polysub(pa, [yt[a]]) ** 1 for a, pa in enumerate(poly))
        gg = np.zeros(2 * p)
        for a in range(3):
            pa = np.polynomial.polynomial.polysub(poly[a], [yt[a]])
            gg[:2 * len(pa) - 1] += np.polynomial.polynomial.polymul(pa, pa)
        roots = np.polynomial.polynomial.polyroots(np.trim_zeros(gg, "b"))
        assert np.min(np.abs(roots - t0)) < 1e-10
        del g


def test_near_list_matches_definition(oracle_lib):
    """near iff |x_t - c_P| <= R_P + eta d_P (c_P vertex mean, R_P max distance to nodes
    and vertices, d_P longest vertex-to-vertex edge), plus self pairs."""
    O = oracle_lib
    d, tg = W.star1280(4, 300)
    tg = W.concat_targets(tg, W.Targets(d.xyz[:50], d.nrm[:50], np.arange(50)))
    osf = O.OracleSurface(d)
    offs, pairs = osf.near(tg)
    V = W.patch_vertices(d)
    c = V.mean(1)
    L = np.max(np.stack([np.linalg.norm(V[:, (k + 1) % 3] - V[:, k], axis=1) for k in range(3)], 1), 1)
    xn = d.xyz.reshape(d.npatch, -1, 3)
    Rp = np.maximum(np.linalg.norm(xn - c[:, None], axis=2).max(1), np.linalg.norm(V - c[:, None], axis=2).max(1))
    for t in range(tg.n):
        dist = np.linalg.norm(tg.xyz[t] - c, axis=1)
        ref = set(np.nonzero(dist <= Rp + L)[0].tolist())
        if tg.self_node[t] >= 0:
            ref.add(int(d.patch_of_node[tg.self_node[t]]))
        got = pairs[offs[t]:offs[t + 1]]
        assert list(got) == sorted(ref)


def test_solid_angle_near_curved_patches(oracle_lib):
    """Omega_0 from the line integrals (eq. solidangle, with the sign of reading R2)
    equals minus the brute-force solid angle int (r'-r).nu/|r'-r|^3 da for targets
    10^-1 .. 10^-4 h above and below curved patches of a star surface.  The vector u of
    Thm. dlp1form must give a half-line from the target that misses the patch; a u
    picked by the smallest u.(r'-r)/|r'-r| over nodes and edge samples alone points
    through the patch for about one such target in five (Omega_0 then off by 4 pi)."""
    O = oracle_lib
    d = W.discretize(W.star_surface(2), 6)
    osf = O.OracleSurface(d)
    V = W.patch_vertices(d)
    rng = np.random.default_rng(3)
    for i in range(8):
        P = int(rng.integers(d.npatch))
        info = osf.patch_internals(P)
        X = _patch_map(d, P, info)
        uv = rng.dirichlet([1, 1, 1])[:2]
        pt, cr = X(uv[None])
        h = np.linalg.norm(V[P][1] - V[P][0])
        k = 1 + (i % 4)
        sgn = 1 if (i // 4) % 2 == 0 else -1
        yt = pt[0] + sgn * 10.0 ** (-k) * h * info["s"] * cr[0] / np.linalg.norm(cr[0])
        xt = info["c"] + (info["R"] @ yt) / info["s"]

        def integrand(uvq, pts, crq):
            dv = yt[None, :] - pts
            return (np.einsum("ia,ia->i", dv, crq) / np.linalg.norm(dv, axis=1) ** 3)[:, None]
        ref = brute.curved_patch(integrand, X, yt, n=12, size_ratio=2.0)[0]
        om0 = osf.pair_B(P, xt, np.array([0.0, 0.0, 1.0]))["Om"][0]
        assert abs(om0 + ref) < 1e-10, (i, P, k, sgn, om0, -ref)
