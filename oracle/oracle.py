"""ctypes loader for the CPU oracle (rrq_oracle.c).

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline leg of
the benchmark import this module.  The product path (the CUDA library and its
binding) never does.

The C source is compiled twice: the FP64 oracle (IEEE binary64 arithmetic) and, from
the same source with -DORC_F128, an IEEE binary128 build of the same algorithm.  Both
take and return binary64 arrays.  The binary128 build is the truth reference for the
binary64 results: where a binary64 row differs from it, the difference is rounding (the
algorithm and its discretisation are the same), so it measures how many digits of the
RRQ row a binary64 implementation keeps.  Select it with ``ext=True``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librrq_oracle.so")
_SO_EXT = os.path.join(_BUILD, "librrq_oracle_f128.so")
_SRC = os.path.join(_HERE, "rrq_oracle.c")
PMAX = 14
KERNELS = ("S", "D", "SP", "DP")
MASK = {"S": 1, "D": 2, "SP": 4, "DP": 8}
_lock = threading.Lock()
_libs = {}


def _compile(so: str, defines, force: bool) -> str:
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", *defines,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


def build(force: bool = False, ext: bool | None = None) -> str:
    """Compile the oracle with gcc (-O2, OpenMP): the binary64 build, and the binary128
    build as well unless ext is False.  Returns the path of the build selected by ext
    (binary64 when ext is None or False)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _compile(_SO, [], force) if not ext else None
    if ext is None or ext:
        so_ext = _compile(_SO_EXT, ["-DORC_F128"], force)
        if ext:
            return so_ext
    return so


class _Opts(C.Structure):
    _fields_ = [("ptilde", C.c_int), ("rho0", C.c_double), ("newton_max", C.c_int),
                ("eta", C.c_double)]


def lib(ext: bool = False):
    """The binary64 oracle, or with ext=True its binary128 build."""
    with _lock:
        L = _libs.get(ext)
        if L is None:
            L = C.CDLL(build(ext=ext))
            L.orc_surface_create.restype = C.c_void_p
            L.orc_surface_destroy.argtypes = [C.c_void_p]
            L.orc_T.restype = C.c_double
            L.orc_patch_kappa.restype = C.c_double
            for name in ("orc_near", "orc_rows", "orc_patch_internals", "orc_edge_root",
                         "orc_pair_B", "orc_patch_bounds", "orc_real_kind"):
                getattr(L, name).restype = C.c_int
            assert L.orc_real_kind() == (1 if ext else 0)
            _libs[ext] = L
    return L


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleSurface:
    """Holds a surface for the oracle.  Arrays are kept alive by this object."""

    def __init__(self, disc, ptilde: int = 0, rho0: float = 0.0, newton_max: int = 0,
                 eta: float = 0.0, ext: bool = False):
        L = self._L = lib(ext)
        self.ext = ext
        self.d = disc
        self.order = np.ascontiguousarray(disc.order, dtype=np.int32)
        self.node_off = np.ascontiguousarray(disc.node_off, dtype=np.int64)
        self.xyz = np.ascontiguousarray(disc.xyz, dtype=np.float64)
        self.nrm = np.ascontiguousarray(disc.nrm, dtype=np.float64)
        self.wts = np.ascontiguousarray(disc.wts, dtype=np.float64)
        self._uv = {p: np.ascontiguousarray(uv, dtype=np.float64) for p, uv in disc.ref_uv.items()}
        arr = (C.c_void_p * (PMAX + 1))()
        for p, uv in self._uv.items():
            arr[p] = uv.ctypes.data
        self._arr = arr
        self.opts = _Opts(ptilde, rho0, newton_max, eta)
        self.h = L.orc_surface_create(C.c_int(disc.npatch), _p(self.order), _p(self.node_off),
                                      _p(self.xyz), _p(self.nrm), _p(self.wts), arr,
                                      C.byref(self.opts))
        if not self.h:
            raise RuntimeError("oracle surface creation failed")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._L.orc_surface_destroy(C.c_void_p(self.h))
                self.h = None
        except Exception:
            pass

    # --------------------------------------------------------------- near lists
    def near(self, targets, tsel=None):
        """Near patches per selected target: (rowptr (nsel+1), patches)."""
        nt = targets.n
        tsel = np.arange(nt, dtype=np.int64) if tsel is None else np.ascontiguousarray(tsel, np.int64)
        txyz = np.ascontiguousarray(targets.xyz, np.float64)
        tself = np.ascontiguousarray(targets.self_node, np.int64)
        counts = np.zeros(len(tsel), np.int64)
        L = self._L
        L.orc_near(C.c_void_p(self.h), C.c_int64(len(tsel)), _p(tsel), _p(txyz), _p(tself),
                   _p(counts), None, None)
        offs = np.zeros(len(tsel) + 1, np.int64)
        np.cumsum(counts, out=offs[1:])
        pairs = np.zeros(max(1, int(offs[-1])), np.int32)
        L.orc_near(C.c_void_p(self.h), C.c_int64(len(tsel)), _p(tsel), _p(txyz), _p(tself),
                   _p(counts), _p(offs), _p(pairs))
        return offs, pairs[: offs[-1]]

    # ------------------------------------------------------------------- rows
    def rows(self, targets, pair_t, pair_P, kernels=KERNELS):
        """Correction rows for explicit pairs: dict kernel -> (npair, n_p) array (uniform p)."""
        pair_t = np.ascontiguousarray(pair_t, np.int64)
        pair_P = np.ascontiguousarray(pair_P, np.int32)
        npair = len(pair_t)
        npn = (self.node_off[1:] - self.node_off[:-1])[pair_P] if npair else np.zeros(0, np.int64)
        val_off = np.zeros(npair, np.int64)
        if npair:
            val_off[1:] = np.cumsum(npn)[:-1]
        tot = int(npn.sum()) if npair else 0
        mask = 0
        for k in kernels:
            mask |= MASK[k]
        vals = {k: np.zeros(max(tot, 1)) for k in KERNELS}
        flags = np.zeros(max(npair, 1), np.int32)
        L = self._L
        r = L.orc_rows(C.c_void_p(self.h), C.c_int64(npair), _p(pair_t), _p(pair_P),
                       _p(np.ascontiguousarray(targets.xyz, np.float64)),
                       _p(np.ascontiguousarray(targets.nrm, np.float64)),
                       _p(np.ascontiguousarray(targets.self_node, np.int64)), C.c_uint(mask),
                       _p(val_off), _p(vals["S"]), _p(vals["D"]), _p(vals["SP"]), _p(vals["DP"]),
                       _p(flags))
        if r != 0:
            raise RuntimeError("oracle rows failed (singular fit)")
        return {k: vals[k][:tot] for k in kernels}, val_off, flags[:npair]

    def csr_rows(self, targets, tsel=None, kernels=KERNELS):
        """CSR restricted to the selected target rows: (rowptr, col, {kernel: val}, flags)."""
        offs, pairs = self.near(targets, tsel)
        tsel = np.arange(targets.n) if tsel is None else np.asarray(tsel)
        pair_t = np.repeat(tsel, np.diff(offs))
        vals, val_off, flags = self.rows(targets, pair_t, pairs, kernels)
        npn = self.node_off[1:] - self.node_off[:-1]
        rowlen = np.zeros(len(tsel), np.int64)
        np.add.at(rowlen, np.repeat(np.arange(len(tsel)), np.diff(offs)), npn[pairs])
        rowptr = np.zeros(len(tsel) + 1, np.int64)
        np.cumsum(rowlen, out=rowptr[1:])
        col = np.concatenate([np.arange(self.node_off[P], self.node_off[P + 1]) for P in pairs]).astype(np.int32) \
            if len(pairs) else np.zeros(0, np.int32)
        return rowptr, col, vals, flags

    # -------------------------------------------------------------- internals
    def patch_internals(self, P: int):
        p = int(self.order[P])
        npn = p * (p + 1) // 2
        pt = self.opts.ptilde if self.opts.ptilde > 0 else 2 * p
        out = dict(frame=np.zeros(13), vert=np.zeros(9), y=np.zeros(npn * 3), ea=np.zeros(9 * p),
                   ey=np.zeros(9 * pt), et=np.zeros(9 * pt), XD=np.zeros(4 * npn * npn),
                   XSp=np.zeros(4 * npn * npn), XS1=np.zeros(npn * npn), XS2=np.zeros(4 * npn * npn))
        r = self._L.orc_patch_internals(C.c_void_p(self.h), C.c_int(P), *[_p(out[k]) for k in
                                      ("frame", "vert", "y", "ea", "ey", "et", "XD", "XSp", "XS1", "XS2")])
        out["status"] = r
        out["c"] = out["frame"][:3]
        out["R"] = out["frame"][3:12].reshape(3, 3)
        out["s"] = out["frame"][12]
        out["vert"] = out["vert"].reshape(3, 3)
        out["y"] = out["y"].reshape(npn, 3)
        out["ea"] = out["ea"].reshape(3, p, 3)
        out["ey"] = out["ey"].reshape(3, pt, 3)
        out["et"] = out["et"].reshape(3, pt, 3)
        for k in ("XD", "XSp", "XS2"):
            out[k] = out[k].reshape(4 * npn, npn)
        out["XS1"] = out["XS1"].reshape(npn, npn)
        return out

    def patch_kappa(self, P: int) -> float:
        """1-norm condition number of patch P's fit matrix A (Sec. 5.1)."""
        return float(self._L.orc_patch_kappa(C.c_void_p(self.h), C.c_int(P)))

    def pair_B(self, P: int, xt, nt, self_i: int = -1):
        p = int(self.order[P])
        npn = p * (p + 1) // 2
        B, dB, Psi, Om, dOm = np.zeros(4 * npn), np.zeros(4 * npn), np.zeros(npn), np.zeros(4), np.zeros(4)
        fl = self._L.orc_pair_B(C.c_void_p(self.h), C.c_int(P), _p(np.ascontiguousarray(xt, np.float64)),
                              _p(np.ascontiguousarray(nt, np.float64)), C.c_int(self_i),
                              _p(B), _p(Psi), _p(dB), _p(Om), _p(dOm))
        return dict(B=B.reshape(npn, 4), Psi=Psi, dB=dB.reshape(npn, 4), Om=Om, dOm=dOm, flags=fl)

    def edge_root(self, P: int, e: int, yt):
        t0 = np.zeros(2)
        c = self._L.orc_edge_root(C.c_void_p(self.h), C.c_int(P), C.c_int(e),
                                _p(np.ascontiguousarray(yt, np.float64)), _p(t0))
        return complex(t0[0], t0[1]), bool(c)


# ------------------------------------------------------------------ free functions

def solid_S(L: int, y, ext: bool = False) -> np.ndarray:
    out = np.zeros(2 * (L + 1) ** 2)
    lib(ext).orc_solid_S(C.c_int(L), _p(np.ascontiguousarray(y, np.float64)), _p(out))
    return out[0::2] + 1j * out[1::2]


def solid_R(L: int, xyz, ext: bool = False) -> np.ndarray:
    out = np.zeros(2 * (L + 1) ** 2)
    lib(ext).orc_solid_R(C.c_int(L), _p(np.ascontiguousarray(xyz, np.float64)), _p(out))
    return out[0::2] + 1j * out[1::2]


def grad_hess_S(L: int, y, l: int, m: int, ext: bool = False):
    g, H = np.zeros(6), np.zeros(18)
    lib(ext).orc_grad_hess_S(C.c_int(L), _p(np.ascontiguousarray(y, np.float64)), C.c_int(l), C.c_int(m),
                          _p(g), _p(H))
    return g[0::2] + 1j * g[1::2], (H[0::2] + 1j * H[1::2]).reshape(3, 3)


def hidx(n: int, q: int) -> int:
    return n * n + n + q


def T(j, k, l, m, ext: bool = False) -> float:
    return lib(ext).orc_T(C.c_int(j), C.c_int(k), C.c_int(l), C.c_int(m))


def gauss_legendre(n: int, ext: bool = False):
    x, w = np.zeros(n), np.zeros(n)
    lib(ext).orc_gauss_legendre(C.c_int(n), _p(x), _p(w))
    return x, w


def ssq_moments(n: int, a: float, b: float, ext: bool = False):
    J, K = np.zeros(n), np.zeros(n)
    lib(ext).orc_ssq_moments(C.c_int(n), C.c_double(a), C.c_double(b), _p(J), _p(K))
    return J, K


def ssq_weights(pt: int, a: float, b: float, ext: bool = False):
    """Singularity-swap weights (m = 1, 3) at the pt Gauss-Legendre nodes for t0 = a + i b."""
    l1, l3 = np.zeros(pt), np.zeros(pt)
    if lib(ext).orc_ssq_weights(C.c_int(pt), C.c_double(a), C.c_double(b), _p(l1), _p(l3)):
        raise ValueError("bad arguments")
    return l1, l3


def bernstein_rho(z: complex, ext: bool = False) -> float:
    r = C.c_double()
    lib(ext).orc_bernstein_rho(C.c_double(z.real), C.c_double(z.imag), C.byref(r))
    return r.value


def lu_solve(A, B, ext: bool = False):
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64).copy()
    nrhs = 1 if B.ndim == 1 else B.shape[1]
    r = lib(ext).orc_lu_solve(C.c_int(A.shape[0]), _p(A), C.c_int(nrhs), _p(B))
    if r:
        raise np.linalg.LinAlgError("singular")
    return B


def basis_batch(p: int, y, ext: bool = False):
    """H^{(l,m)} and grad H^{(l,m)} (1 <= m <= l <= p) at points y (n, 3)."""
    y = np.ascontiguousarray(y, np.float64).reshape(-1, 3)
    npn = p * (p + 1) // 2
    H = np.zeros((len(y), npn))
    gH = np.zeros((len(y), npn, 3))
    lib(ext).orc_basis_batch(C.c_int(p), C.c_int64(len(y)), _p(y), _p(H), _p(gH))
    return H, gH
