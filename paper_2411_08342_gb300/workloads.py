"""Seeded synthetic inputs: reference nodes, triangulated surfaces, targets, densities.

This module holds geometry and input generation only.  It contains none of the
quadrature method's arithmetic (no harmonic fit, no line integrals, no weights
of the correction), so the CUDA path and the CPU oracle can both be fed from it.

Conventions shared by every surface produced here:

* Reference triangle T with vertices (0,0), (1,0), (0,1).  A patch is the map
  X(u,v) of T into R^3; its orientation X_u x X_v is the outward normal.
* Each patch of order p carries n_p = p(p+1)/2 nodes (the paper's node count,
  Sec. 3.2, eq. (dlpdensitylinearsystem2)): the images X(u_i, v_i) of the
  reference nodes below.
* Reference nodes: the Blyth-Pozrikidis blend of 1-D Gauss-Legendre points
  (nodes strictly inside T, unisolvent for total degree p-1).  The paper uses
  Vioreanu-Rokhlin nodes (Sec. 5); any unisolvent interior set serves.
* Smooth weights: interpolatory weights of the node set on T times the area
  element |X_u x X_v| at the node; node normals are unit(X_u x X_v) of the exact
  surface, differentiated by complex step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Reference nodes and weights on T
# ----------------------------------------------------------------------------


def gauss_legendre_01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def ref_nodes(p: int) -> np.ndarray:
    """(n_p, 2) reference nodes (u, v) for order p (degree p-1 interpolation)."""
    if p < 1:
        raise ValueError("order p must be >= 1")
    n = p - 1
    g, _ = gauss_legendre_01(p)
    pts = []
    for i in range(n + 1):
        for j in range(n + 1 - i):
            k = n - i - j
            l1 = (1.0 + 2.0 * g[j] - g[i] - g[k]) / 3.0
            l2 = (1.0 + 2.0 * g[k] - g[i] - g[j]) / 3.0
            pts.append((l1, l2))
    return np.ascontiguousarray(np.array(pts, dtype=np.float64))


def _dubiner(uv: np.ndarray, deg: int) -> np.ndarray:
    """Orthogonal (Koornwinder-Dubiner) basis of total degree <= deg at uv."""
    u, v = uv[:, 0], uv[:, 1]
    x = 2.0 * u - 1.0 + v
    w = 1.0 - v
    eta = 2.0 * v - 1.0
    # homogenised Legendre L_a = w^a P_a(x / w)
    L = [np.ones_like(u), x.copy()]
    for a in range(1, deg):
        L.append(((2 * a + 1) * x * L[a] - a * w * w * L[a - 1]) / (a + 1))
    cols = []
    for a in range(deg + 1):
        al = 2 * a + 1
        # Jacobi P_b^{(al,0)}(eta)
        J = [np.ones_like(u)]
        if deg - a >= 1:
            J.append(0.5 * ((al + 2) * eta + al))
        for b in range(1, deg - a):
            c1 = 2 * (b + 1) * (b + al + 1) * (2 * b + al)
            c2 = (2 * b + al + 1) * (al * al)
            c3 = (2 * b + al) * (2 * b + al + 1) * (2 * b + al + 2)
            c4 = 2 * (b + al) * b * (2 * b + al + 2)
            J.append(((c2 + c3 * eta) * J[b] - c4 * J[b - 1]) / c1)
        for b in range(deg - a + 1):
            cols.append(L[a] * J[b])
    return np.array(cols).T


def interp_matrix(ref_uv: np.ndarray, p: int, uv: np.ndarray) -> np.ndarray:
    """Rows: Lagrange basis of the reference nodes evaluated at uv (m, n_p)."""
    V = _dubiner(ref_uv, p - 1)
    Vq = _dubiner(np.atleast_2d(uv), p - 1)
    return np.linalg.solve(V.T, Vq.T).T


def ref_weights(p: int) -> np.ndarray:
    """Interpolatory weights of ref_nodes(p) on T (exact for degree p-1): V^T w = m in the
    orthogonal Koornwinder-Dubiner basis, whose moments over T are 1/2 for the constant
    and 0 otherwise.  (The monomial basis would make V ill-conditioned: cond ~ 5e10 at
    p = 12, weights wrong by ~1e-7.)"""
    uv = ref_nodes(p)
    V = _dubiner(uv, p - 1)
    mom = np.zeros(V.shape[1])
    mom[0] = 0.5
    return np.linalg.solve(V.T, mom)


def n_nodes(p: int) -> int:
    return p * (p + 1) // 2


# ----------------------------------------------------------------------------
# Real spherical harmonics (paper normalisation eq. (ylmdef), no Condon-Shortley
# phase), written as real polynomials of a unit vector so they are complex-step
# friendly.
# ----------------------------------------------------------------------------


def _dmlegendre(l: int, m: int, z):
    """d^m/dz^m P_l(z) via the power-series of P_l (exact polynomial)."""
    # P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^(l-2k)
    out = 0.0 * z
    for k in range(l // 2 + 1):
        e = l - 2 * k
        if e < m:
            continue
        c = (-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l) / 2.0**l
        c *= math.factorial(e) / math.factorial(e - m)
        out = out + c * z ** (e - m)
    return out


def real_ylm(l: int, m: int, xyz, part: str = "re"):
    """Re or Im of Y_l^m(x_hat) (paper normalisation) for unit vectors xyz (..., 3)."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    c, s = 1.0 + 0.0 * x, 0.0 * x
    for _ in range(m):
        c, s = x * c - y * s, x * s + y * c
    norm = math.sqrt(2 * l + 1) * math.sqrt(math.factorial(l - m) / math.factorial(l + m))
    d = _dmlegendre(l, m, z)
    return norm * d * (c if part == "re" else s)


# ----------------------------------------------------------------------------
# Surfaces
# ----------------------------------------------------------------------------


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1)[:, None]
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    return v, f


def icosphere_flat(levels: int):
    """Flat triangles (nf, 3, 3) of an icosahedron split 4-fold `levels` times,
    vertices on the unit sphere, oriented counter-clockwise seen from outside."""
    v, f = _icosahedron()
    tris = v[f]
    for _ in range(levels):
        a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
        ab = (a + b) / 2
        bc = (b + c) / 2
        ca = (c + a) / 2
        ab /= np.linalg.norm(ab, axis=1)[:, None]
        bc /= np.linalg.norm(bc, axis=1)[:, None]
        ca /= np.linalg.norm(ca, axis=1)[:, None]
        tris = np.concatenate([np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
                               np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)], 0)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    flip = np.einsum("ij,ij->i", n, tris.sum(1)) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def _cnorm(x):
    return np.sqrt(x[..., 0] * x[..., 0] + x[..., 1] * x[..., 1] + x[..., 2] * x[..., 2])


@dataclass
class Surface:
    """A triangulated surface: each patch maps T -> R^3 through `patch_map`."""
    name: str
    npatch: int
    patch_map: callable  # (patch indices (k,), uv (k, m, 2) complex-ok) -> (k, m, 3)
    meta: dict = field(default_factory=dict)


def _flat_patch_map(tris, radial):
    def fmap(idx, uv):
        tr = tris[idx]
        a = tr[:, None, 0, :]
        x = a + uv[..., 0:1] * (tr[:, None, 1, :] - a) + uv[..., 1:2] * (tr[:, None, 2, :] - a)
        return radial(x)
    return fmap


def sphere_surface(levels: int) -> Surface:
    tris = icosphere_flat(levels)
    return Surface(f"sphere{len(tris)}", len(tris),
                   _flat_patch_map(tris, lambda x: x / _cnorm(x)[..., None]))


def star_surface(levels: int, terms=((3, 2, 0.2), (5, 1, 0.1))) -> Surface:
    """r(theta, phi) = 1 + sum a * Re Y_l^m over an icosahedral mesh (radial map)."""
    tris = icosphere_flat(levels)

    def radial(x):
        xh = x / _cnorm(x)[..., None]
        r = 1.0
        for (l, m, a) in terms:
            r = r + a * real_ylm(l, m, xh, "re")
        return xh * r[..., None]
    return Surface(f"star{len(tris)}", len(tris), _flat_patch_map(tris, radial),
                   {"terms": list(terms)})


def ellipsoid_surface(levels: int, axes=(2.0, 1.0, 0.5)) -> Surface:
    tris = icosphere_flat(levels)
    ax = np.array(axes)
    return Surface(f"ellipsoid{len(tris)}", len(tris),
                   _flat_patch_map(tris, lambda x: x / _cnorm(x)[..., None] * ax))


def wavy_torus_surface(n_theta: int, n_phi: int, R=1.0, r0=0.35, amp=0.05) -> Surface:
    """Torus with tube radius r0 + amp cos(5 phi) sin(3 theta); 2 triangles per
    cell of an n_theta x n_phi parameter grid (phi toroidal, theta poloidal)."""
    cells = []
    for i in range(n_phi):
        for j in range(n_theta):
            p00 = (i, j)
            p10 = (i + 1, j)
            p01 = (i, j + 1)
            p11 = (i + 1, j + 1)
            cells.append((p00, p10, p11))
            cells.append((p00, p11, p01))
    par = np.array(cells, dtype=np.float64)
    par[..., 0] *= 2 * math.pi / n_phi
    par[..., 1] *= 2 * math.pi / n_theta

    def fmap(idx, uv):
        tr = par[idx]
        a = tr[:, None, 0, :]
        q = a + uv[..., 0:1] * (tr[:, None, 1, :] - a) + uv[..., 1:2] * (tr[:, None, 2, :] - a)
        ph, th = q[..., 0], q[..., 1]
        rr = r0 + amp * np.cos(5 * ph) * np.sin(3 * th)
        # (phi, theta) with this orientation gives an outward X_u x X_v
        return np.stack([(R + rr * np.cos(th)) * np.cos(ph),
                         (R + rr * np.cos(th)) * np.sin(ph),
                         rr * np.sin(th)], -1)
    return Surface(f"torus{len(par)}", len(par), fmap, {"n_theta": n_theta, "n_phi": n_phi})


# Stellarator of Sec. 5 (eq. stellarator): non-zero coefficients delta_{i,j}
STELLARATOR_DELTA = {(-1, -1): 0.17, (-1, 0): 0.11, (0, 0): 1.0, (1, 0): 4.5, (2, 0): -0.25, (0, 1): 0.07,
                     (2, 1): -0.45}


def _stellarator_xyz(u, v):
    x = y = z = 0.0
    for (i, j), dl in STELLARATOR_DELTA.items():
        ang = (1 - i) * u + j * v
        x = x + dl * np.cos(v) * np.cos(ang)
        y = y + dl * np.sin(v) * np.cos(ang)
        z = z + dl * np.sin(ang)
    return np.stack([x, y, z], -1)


def stellarator_surface(n_u: int, n_v: int) -> Surface:
    """The stellarator r(u, v) of eq. stellarator on [0, 2 pi]^2, the parameter square cut
    into n_u x n_v equal rectangles of two triangles each; triangles oriented so that
    X_u x X_v points out of the enclosed volume."""
    def build(flip):
        cells = []
        for i in range(n_u):
            for j in range(n_v):
                p00, p10, p01, p11 = (i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)
                if flip:
                    cells += [(p00, p11, p10), (p00, p01, p11)]
                else:
                    cells += [(p00, p10, p11), (p00, p11, p01)]
        par = np.array(cells, dtype=np.float64)
        par[..., 0] *= 2 * math.pi / n_u
        par[..., 1] *= 2 * math.pi / n_v

        def fmap(idx, uv):
            tr = par[idx]
            a = tr[:, None, 0, :]
            q = a + uv[..., 0:1] * (tr[:, None, 1, :] - a) + uv[..., 1:2] * (tr[:, None, 2, :] - a)
            return _stellarator_xyz(q[..., 0], q[..., 1])
        return Surface(f"stellarator{len(par)}", len(par), fmap, {"n_u": n_u, "n_v": n_v})
    surf = build(False)
    # enclosed volume by the divergence theorem, (1/3) int x . n dA, on a coarse rule
    d = discretize(surf, 2)
    if np.sum(np.einsum("ia,ia->i", d.xyz, d.nrm) * d.wts) < 0:
        surf = build(True)
    return surf


def stellarator(p: int = 6, n_u: int = 24, n_v: int = 72):
    """Stellarator surface with all on-surface nodes as targets (the points of the
    paper's throughput table)."""
    d = discretize(stellarator_surface(n_u, n_v), p)
    return d, on_surface_targets(d)


def paraboloid_patch(H: float, h: float = 1.0) -> Surface:
    """One patch of the paraboloid r(u, v) = (u, v, H (u^2 + v^2) / 2) over the equilateral
    triangle of side h centred at the origin of the (u, v) plane (Sec. 5.1, eq. paraboloid);
    its largest mean curvature, H, is reached at the origin."""
    R = h / math.sqrt(3.0)
    ang = 0.5 * math.pi + 2.0 * math.pi * np.arange(3) / 3.0
    tri = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros(3)], -1)[None]

    def lift(x):
        return np.stack([x[..., 0], x[..., 1], 0.5 * H * (x[..., 0] ** 2 + x[..., 1] ** 2)], -1)
    return Surface(f"paraboloid_H{H:g}_h{h:g}", 1, _flat_patch_map(tri, lift), {"H": H, "h": h})


def flat_surface(tris: np.ndarray) -> Surface:
    """Planar triangles (k, 3, 3), mapped affinely."""
    tris = np.asarray(tris, dtype=np.float64)
    return Surface(f"flat{len(tris)}", len(tris), _flat_patch_map(tris, lambda x: x))


# ----------------------------------------------------------------------------
# Discretisation
# ----------------------------------------------------------------------------


@dataclass
class Discretization:
    p: int
    npatch: int
    order: np.ndarray      # (npatch,) int32
    node_off: np.ndarray   # (npatch+1,) int64
    xyz: np.ndarray        # (N, 3)
    nrm: np.ndarray        # (N, 3)
    wts: np.ndarray        # (N,)
    ref_uv: dict           # p -> (n_p, 2)
    surface: Surface = None
    patch_of_node: np.ndarray = None

    @property
    def nnode(self) -> int:
        return int(self.node_off[-1])


def _map_with_jacobian(surf: Surface, idx: np.ndarray, uv: np.ndarray):
    """Positions, unit normals and area elements via complex-step derivatives."""
    h = 1e-30
    X = surf.patch_map(idx, uv.astype(np.complex128)).real
    du = np.zeros_like(uv, dtype=np.complex128)
    du[..., 0] = 1j * h
    Xu = surf.patch_map(idx, uv + du).imag / h
    dv = np.zeros_like(uv, dtype=np.complex128)
    dv[..., 1] = 1j * h
    Xv = surf.patch_map(idx, uv + dv).imag / h
    n = np.cross(Xu, Xv)
    J = np.linalg.norm(n, axis=-1)
    return X, n / J[..., None], J


def discretize(surf: Surface, p: int) -> Discretization:
    uv = ref_nodes(p)
    W = ref_weights(p)
    npn = len(uv)
    idx = np.arange(surf.npatch)
    X, nrm, J = _map_with_jacobian(surf, idx, np.broadcast_to(uv, (surf.npatch, npn, 2)).copy())
    return Discretization(
        p=p, npatch=surf.npatch,
        order=np.full(surf.npatch, p, dtype=np.int32),
        node_off=(np.arange(surf.npatch + 1, dtype=np.int64) * npn),
        xyz=np.ascontiguousarray(X.reshape(-1, 3)),
        nrm=np.ascontiguousarray(nrm.reshape(-1, 3)),
        wts=np.ascontiguousarray((J * W[None, :]).reshape(-1)),
        ref_uv={p: uv}, surface=surf,
        patch_of_node=np.repeat(idx, npn).astype(np.int64))


@dataclass
class Targets:
    xyz: np.ndarray        # (T, 3)
    nrm: np.ndarray        # (T, 3)
    self_node: np.ndarray  # (T,) int64, -1 if not a surface node

    @property
    def n(self) -> int:
        return len(self.xyz)


def on_surface_targets(d: Discretization) -> Targets:
    return Targets(d.xyz.copy(), d.nrm.copy(), np.arange(d.nnode, dtype=np.int64))


def patch_vertices(d: Discretization) -> np.ndarray:
    """(npatch, 3, 3) images of the reference vertices under the node interpolant."""
    M = interp_matrix(d.ref_uv[d.p], d.p, np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]))
    x = d.xyz.reshape(d.npatch, -1, 3)
    return np.einsum("vi,pia->pva", M, x)


def off_surface_targets(d: Discretization, n: int, seed: int, kmax: float = 6.0) -> Targets:
    """Random patch, uniform point of T, pushed along the exterior normal by
    10^-k h with k ~ U[0, kmax] and h the patch's longest vertex-to-vertex chord.
    The base point lies on the node interpolant of the patch."""
    rng = np.random.default_rng(seed)
    P = rng.integers(0, d.npatch, n)
    a, b = rng.random(n), rng.random(n)
    swap = a + b > 1
    a[swap], b[swap] = 1 - a[swap], 1 - b[swap]
    uv = np.stack([a, b], -1)
    k = rng.random(n) * kmax
    V = patch_vertices(d)
    h = np.max(np.stack([np.linalg.norm(V[:, 1] - V[:, 0], axis=1),
                         np.linalg.norm(V[:, 2] - V[:, 1], axis=1),
                         np.linalg.norm(V[:, 0] - V[:, 2], axis=1)], 1), axis=1)
    M = interp_matrix(d.ref_uv[d.p], d.p, uv)              # (n, n_p)
    x = d.xyz.reshape(d.npatch, -1, 3)[P]                   # (n, n_p, 3)
    base = np.einsum("ti,tia->ta", M, x)
    _, nrm, _ = _map_with_jacobian(d.surface, P, uv[:, None, :])
    nrm = nrm[:, 0, :]
    xyz = base + (10.0 ** (-k) * h[P])[:, None] * nrm
    return Targets(np.ascontiguousarray(xyz), np.ascontiguousarray(nrm),
                   np.full(n, -1, dtype=np.int64))


def concat_targets(*ts: Targets) -> Targets:
    return Targets(np.concatenate([t.xyz for t in ts]), np.concatenate([t.nrm for t in ts]),
                   np.concatenate([t.self_node for t in ts]))


def random_ylm_density(xyz: np.ndarray, lmax: int, seed: int) -> np.ndarray:
    """sum over l <= lmax of N(0,1) coefficients times Re/Im Y_l^m of the direction."""
    rng = np.random.default_rng(seed)
    xh = xyz / np.linalg.norm(xyz, axis=1)[:, None]
    out = np.zeros(len(xyz))
    for l in range(lmax + 1):
        for m in range(l + 1):
            out += rng.standard_normal() * real_ylm(l, m, xh, "re")
            if m > 0:
                out += rng.standard_normal() * real_ylm(l, m, xh, "im")
    return out


# ----------------------------------------------------------------------------
# Named workloads (sizes in the paper's convention n_p = p(p+1)/2)
# ----------------------------------------------------------------------------

WORKLOAD_SEED = 20241113


def sphere80(p: int = 4):
    """Unit sphere, icosahedron split once (80 patches), all on-surface nodes."""
    d = discretize(sphere_surface(1), p)
    return d, on_surface_targets(d)


def star1280(p: int = 6, ntarg: int = 200_000, seed: int = WORKLOAD_SEED + 2):
    """Star surface r = 1 + 0.2 Re Y_3^2 + 0.1 Re Y_5^1 on 1280 patches, with
    off-surface targets at 10^-k h, k ~ U[0,6]."""
    d = discretize(star_surface(3), p)
    return d, off_surface_targets(d, ntarg, seed)


def wavy_torus(p: int = 8, n_theta: int = 64, n_phi: int = 160, noff: int = 200_000,
               seed: int = WORKLOAD_SEED + 3):
    d = discretize(wavy_torus_surface(n_theta, n_phi), p)
    return d, concat_targets(on_surface_targets(d), off_surface_targets(d, noff, seed))


def ellipsoid81920(p: int = 6, levels: int = 6):
    d = discretize(ellipsoid_surface(levels), p)
    return d, on_surface_targets(d)


def random_star_terms(rng, lmin: int = 2, lmax: int = 6, amp: float = 0.25):
    """Terms (l, m, a) of r = 1 + sum a Re Y_l^m, lmin <= l <= lmax, 0 <= m <= l, with
    a ~ N(0,1) rescaled so that the largest |perturbation| on a 64 x 128 (theta, phi)
    grid is amp."""
    terms = [(l, m, rng.standard_normal()) for l in range(lmin, lmax + 1) for m in range(l + 1)]
    th, ph = np.meshgrid(np.linspace(0, np.pi, 64), np.linspace(0, 2 * np.pi, 128, endpoint=False), indexing="ij")
    xh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    pert = sum(a * real_ylm(l, m, xh, "re") for (l, m, a) in terms)
    s = amp / np.abs(pert).max()
    return [(l, m, a * s) for (l, m, a) in terms]


def star_batch(nsurf: int = 64, levels=(1, 2, 3, 4), orders=(4, 6, 8), seed: int = WORKLOAD_SEED + 4):
    """Batched workload: nsurf star surfaces with seeded random perturbations (max 0.25),
    each on an icosahedral mesh of 20 * 4^L patches with L drawn from `levels` and an
    order drawn from `orders`; targets are the on-surface nodes."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsurf):
        L = int(rng.choice(levels))
        p = int(rng.choice(orders))
        terms = random_star_terms(rng)
        d = discretize(star_surface(L, terms=tuple(terms)), p)
        out.append((d, on_surface_targets(d)))
    return out
