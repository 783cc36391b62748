"""CPU pins of the rotation-based translation scheme (Sec. 2.3, the remark on fast
translation) that the rotation variant of the per-pair kernel runs: written here from the
mathematics, independently of the CUDA sources, in the device's harmonic normalisation
Rn_l^m = R_l^m / sqrt((l-m)!(l+m)!) (translation coefficients T = 1, Rn^{-m} = (-1)^m
conj(Rn^m)).

* the closed form of the rotation by 90 degrees about Y,
  Delta_{mk} = 2^{-l} sum_s (-1)^{k-m+s} C(l+k, k-m+s) C(l-k, s), against harmonics
  evaluated at rotated points;
* the factorisation Ry(b) = Rz(90) Ry(90) Rz(b) Ry(-90) Rz(-90) that lets two fixed
  tables and phases stand for every rotation;
* rotate / translate along the polar axis / rotate back, with sets held for k >= 0 only and
  the tables folded into their real and imaginary blocks, equals the direct translation
  sums of eqs. l2ltranslation2-3 (weights W_{j,l} per j, as the C_{j,l}, D_{j,l} factors),
  and so does the normal derivative of the translation kernel through its three on-axis
  bands; also for targets at the origin and on the polar axis."""
from math import comb, factorial

import numpy as np
import pytest

P = 7


def rn_table(L, a):
    """Rn_l^m(a) for 0 <= l <= L, |m| <= l: the associated-Legendre recurrence on
    W_l^m = r^l P_l^m e^{i m phi} scaled to unit translation coefficients."""
    X, Y, Z = a
    r2 = X * X + Y * Y + Z * Z
    S = {}
    for m in range(L + 1):
        w = 1.0 + 0j
        for k in range(1, m + 1):
            w = w * (X + 1j * Y) / (2 * k)
        prev, cur = 0j, w
        S[(m, m)] = cur
        for l in range(m, L):
            nxt = ((2 * l + 1) * Z * cur - r2 * prev) / ((l - m + 1) * (l + m + 1))
            S[(l + 1, m)] = nxt
            prev, cur = cur, nxt
    for (l, m) in list(S):
        if m > 0:
            S[(l, -m)] = (-1) ** m * np.conj(S[(l, m)])
    return S


def rz(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def ry(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def delta_plus(l):
    D = np.zeros((2 * l + 1, 2 * l + 1))
    for m in range(-l, l + 1):
        for k in range(-l, l + 1):
            acc = 0
            for s in range(0, l - k + 1):
                a = k - m + s
                if 0 <= a <= l + k:
                    acc += (-1) ** a * comb(l + k, a) * comb(l - k, s)
            D[m + l, k + l] = acc / 2 ** l
    return D


def test_translation_identity_unit_coefficients():
    """Rn_l^m(a + b) = sum_{j,k} Rn_j^k(a) Rn_{l-j}^{m-k}(b): the normalisation the kernel
    uses, with T_{jk,lm} of eq. (tjklmdef) absorbed."""
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=3) * 0.4, rng.normal(size=3) * 0.4
    Sa, Sb, Sab = rn_table(P, a), rn_table(P, b), rn_table(P, a + b)
    for l in range(P + 1):
        for m in range(-l, l + 1):
            s = sum(Sa[(j, k)] * Sb.get((l - j, m - k), 0) for j in range(l + 1) for k in range(-j, j + 1)
                    if abs(m - k) <= l - j)
            assert abs(s - Sab[(l, m)]) < 1e-13 * (1 + abs(Sab[(l, m)]))


def test_delta_is_the_rotation_by_90_degrees_about_y():
    rng = np.random.default_rng(2)
    for _ in range(3):
        a = rng.normal(size=3)
        Sa, Sr = rn_table(P, a), rn_table(P, ry(np.pi / 2) @ a)
        Sm = rn_table(P, ry(-np.pi / 2) @ a)
        for l in range(P + 1):
            D = delta_plus(l)
            va = np.array([Sa[(l, k)] for k in range(-l, l + 1)])
            sign = np.array([[(-1) ** (k - m) for k in range(-l, l + 1)] for m in range(-l, l + 1)])
            assert np.allclose(D @ va, [Sr[(l, m)] for m in range(-l, l + 1)], rtol=1e-12, atol=1e-12)
            assert np.allclose((sign * D) @ va, [Sm[(l, m)] for m in range(-l, l + 1)], rtol=1e-12, atol=1e-12)


def test_y_rotation_through_fixed_tables():
    for b in (0.3, 1.7, -2.4):
        assert np.abs(ry(b) - rz(np.pi / 2) @ ry(np.pi / 2) @ rz(b) @ ry(-np.pi / 2) @ rz(-np.pi / 2)).max() < 1e-15


def folded(D, l):
    """Real and imaginary blocks of D for sets with c_{-k} = (-1)^k conj(c_k)."""
    A = np.zeros((l + 1, l + 1))
    B = np.zeros((l + 1, l + 1))
    for m in range(l + 1):
        A[m, 0] = D[m + l, l]
        for k in range(1, l + 1):
            A[m, k] = D[m + l, k + l] + (-1) ** k * D[m + l, -k + l]
            B[m, k] = D[m + l, k + l] - (-1) ** k * D[m + l, -k + l]
    return A, B


def apply_folded(blk, v, l):
    A, B = blk
    out = np.zeros(l + 1, complex)
    for m in range(l + 1):
        out[m] = A[m] @ v.real + (1j * (B[m, 1:] @ v[1:].imag) if m else 0.0)
    return out


def direct_sums(sets, jmins, W, b, nu):
    """Im of the translated sums for m >= 1 (eqs. l2ltranslation2-3 with a weight W_{j,l}
    per j), and for the sets flagged deriv the normal derivative of the kernel as well."""
    S = rn_table(P, b)

    def full(c, j, k):
        return c[j, k] if k >= 0 else (-1) ** k * np.conj(c[j, -k])

    def grad(n, q):
        if n == 0:
            return np.zeros(3, complex)
        g = lambda qq: S.get((n - 1, qq), 0) if abs(qq) <= n - 1 else 0
        return np.array([(g(q - 1) - g(q + 1)) / 2, 1j * (g(q - 1) + g(q + 1)) / 2, g(q)])

    out = np.zeros((len(sets), P + 1, P + 1))
    for t, (c, jmin, deriv) in enumerate(zip(sets, jmins, [False, True, False])):
        for l in range(1, P + 1):
            for m in range(1, l + 1):
                acc = 0j
                for j in range(jmin, l + 1):
                    for k in range(-j, j + 1):
                        n, q = l - j, m - k
                        if abs(q) > n:
                            continue
                        acc += W[j, l] * S[(n, q)] * full(c, j, k)
                        if deriv:   # the derivative acts on set 0 (Q) beside this set (dQ)
                            acc += W[j, l] * (nu @ grad(n, q)) * full(sets[0], j, k)
                out[t, l, m] = acc.imag
    return out


def rotated_sums(sets, jmins, W, b, nu):
    AP = [folded(delta_plus(l), l) for l in range(P + 1)]
    AM = [folded(np.array([[(-1) ** (k - m) for k in range(-l, l + 1)] for m in range(-l, l + 1)]) *
                 delta_plus(l), l) for l in range(P + 1)]
    rho = np.linalg.norm(b)
    rxy = np.hypot(b[0], b[1])
    cph, sph = (b[0] / rxy, b[1] / rxy) if rxy > 0 else (1.0, 0.0)
    cth, sth = (b[2] / rho, rxy / rho) if rho > 0 else (1.0, 0.0)
    eth = np.array([(cth + 1j * sth) ** k for k in range(P + 1)])
    eph = np.array([(-sph + 1j * cph) ** k for k in range(P + 1)])         # e^{ik(phi + 90)}
    rp = np.array([rho ** n / factorial(n) for n in range(P + 1)])
    x1, y1 = cph * nu[0] + sph * nu[1], cph * nu[1] - sph * nu[0]
    nt = np.array([cth * x1 - sth * nu[2], y1, sth * x1 + cth * nu[2]])   # U nu
    rot = []
    for c, jmin in zip(sets, jmins):
        cp = c.copy()
        for j in range(jmin, P + 1):
            y = apply_folded(AM[j], cp[j, :j + 1] * np.conj(eph[:j + 1]), j) * np.conj(eth[:j + 1])
            cp[j, :j + 1] = apply_folded(AP[j], y, j) * (1j) ** np.arange(j + 1)
        rot.append(cp)

    def cfull(c, j, k):
        return c[j, k] if k >= 0 else (-1) ** k * np.conj(c[j, -k])

    out = np.zeros((len(sets), P + 1, P + 1))
    for t, (jmin, deriv) in enumerate(zip(jmins, [False, True, False])):
        for l in range(1, P + 1):
            O = np.zeros(l + 1, complex)
            for mq in range(l + 1):
                acc = sum(W[j, l] * rp[l - j] * rot[t][j, mq] for j in range(max(jmin, mq), l + 1))
                if deriv:
                    for j in range(jmins[0], l):
                        f = W[j, l] * rp[l - j - 1]
                        for kk, g in ((mq - 1, (nt[0] + 1j * nt[1]) / 2), (mq, nt[2]), (mq + 1, (-nt[0] + 1j * nt[1]) / 2)):
                            if abs(kk) <= j:
                                acc += f * g * cfull(rot[0], j, kk)
                O[mq] = acc * (-1j) ** mq
            u = apply_folded(AP[l], apply_folded(AM[l], O, l) * eth[:l + 1], l)
            for m in range(1, l + 1):
                out[t, l, m] = (eph[m] * u[m]).imag
    return out


@pytest.mark.parametrize("where", ["general", "origin", "plus_axis", "minus_axis"])
def test_rotated_translation_equals_direct_sums(where):
    rng = np.random.default_rng(3)
    W = rng.uniform(0.5, 1.5, size=(P + 1, P + 1))
    jmins = [2, 2, 1]       # Q-like, dQ-like (with the derivative term on the first set), V-like

    def rset(jmin):
        c = np.zeros((P + 1, P + 1), complex)
        for j in range(jmin, P + 1):
            for k in range(j + 1):
                c[j, k] = (rng.normal() + (1j * rng.normal() if k else 0)) * 0.7 ** j / np.sqrt(
                    float(factorial(j - k) * factorial(j + k))) * factorial(j)
        return c
    sets = [rset(j) for j in jmins]
    b = {"general": rng.normal(size=3) * 0.6, "origin": np.zeros(3), "plus_axis": np.array([0.0, 0.0, 0.8]),
         "minus_axis": np.array([0.0, 0.0, -0.8])}[where]
    nu = rng.normal(size=3)
    nu /= np.linalg.norm(nu)
    ref = direct_sums(sets, jmins, W, b, nu)
    got = rotated_sums(sets, jmins, W, b, nu)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= 1e-12 * scale, np.abs(got - ref).max() / scale
