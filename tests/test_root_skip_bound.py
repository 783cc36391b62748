"""The root-finding of the per-pair stage skips Newton for an edge only when a bound shows
that no complex root of sum_a (y_a(t) - y'_a)^2 lies in the singularity-swap ellipse
E_rho0 (the rule then is the upsampled one whatever the root).  This checks the bound,
written out here from the same formula, against the oracle's roots on the coarse curved
star mesh where a plain chord-root estimate misjudges the rule: the bound never skips an
edge whose root lies in E_rho0, while the chord estimate (radius > 1.5 rho0) does."""
import numpy as np

from paper_2411_08342_gb300 import workloads as W


def _bern(z):
    w = z + np.sqrt(z - 1 + 0j) * np.sqrt(z + 1 + 0j)
    r = abs(w)
    return r if r >= 1 else 1 / r


def _check(O, d, tg, npairs, seed=0):
    p = d.p
    osf = O.OracleSurface(d)
    offs, pairs = osf.near(tg)
    pair_t = np.repeat(np.arange(tg.n), np.diff(offs))
    rho0 = 10 ** (5 / (2 * p))
    A0 = 0.5 * (rho0 + 1 / rho0)
    idx = np.random.default_rng(seed).choice(len(pairs), min(npairs, len(pairs)), replace=False)
    info = {}
    skipped = heuristic_wrong = 0
    for n in idx:
        t, P = pair_t[n], pairs[n]
        if P not in info:
            info[P] = osf.patch_internals(P)
        fr = info[P]["frame"]
        yt = fr[12] * (fr[3:12].reshape(3, 3).T @ (tg.xyz[t] - fr[:3]))
        ea = info[P]["ea"].reshape(3, p, 3)
        for e in range(3):
            a = ea[e]
            yp, ym = a.sum(0), (a * ((-1.0) ** np.arange(p))[:, None]).sum(0)
            c, b = 0.5 * (yp + ym), 0.5 * (yp - ym)
            w = yt - c
            bb = b @ b
            tau = complex(b @ w / bb, np.linalg.norm(np.cross(b, w)) / bb)
            rc = _bern(tau)
            D = sum(np.linalg.norm(a[k]) * (rho0 ** k + A0) for k in range(2, p))
            gap = max(0.0, 0.5 * (rc + 1 / rc - rho0 - 1 / rho0))
            skip = tau.imag > 0 and rc > rho0 and bb * gap * gap > 2 * (np.sqrt(bb) * A0 + np.linalg.norm(w)) * D + D * D
            t0, conv = osf.edge_root(P, e, yt)
            inside = conv and _bern(complex(t0.real, abs(t0.imag))) < rho0
            assert not (skip and inside), (t, P, e, t0, rc)
            skipped += skip
            heuristic_wrong += (tau.imag > 0 and rc > 1.5 * rho0 and inside)
    return skipped, heuristic_wrong


def test_root_skip_bound(oracle_lib):
    # 80 strongly curved patches: the chord estimate misjudges edges, the bound never skips wrongly
    p = 6
    d = W.discretize(W.star_surface(1), p)
    rng = np.random.default_rng(100 + p)
    on = W.on_surface_targets(d)
    sel = rng.choice(on.n, 200, replace=False)
    tg = W.concat_targets(W.Targets(on.xyz[sel], on.nrm[sel], on.self_node[sel]),
                          W.off_surface_targets(d, 200, seed=100 + p))
    _, wrong = _check(oracle_lib, d, tg, 2500)
    assert wrong > 0
    # the benchmark mesh (1280 patches): the bound does skip a share of the far edges
    d, tg = W.star1280(6, 2000)
    skipped, _ = _check(oracle_lib, d, tg, 800)
    assert skipped > 0
