"""Thin ctypes binding of librrq (include/rrq.h).

Argument marshalling only: every step of the correction build and of the apply runs
in the CUDA library.  Device arrays are torch CUDA tensors; host arrays are numpy
arrays (used with inputs_on_host=1).  There is no CPU fallback: loading fails loudly
when the library cannot be built or loaded, and every compute call needs a GPU.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PMAX = 14
S, D, SP, DP = 1, 2, 4, 8
KERNEL_BITS = {"S": S, "D": D, "SP": SP, "DP": DP}
KERNEL_SLOT = {"S": 0, "D": 1, "SP": 2, "DP": 3}
_lock = threading.Lock()
_lib = None


class Surface(C.Structure):
    _fields_ = [("npatch", C.c_int32), ("order", C.c_void_p), ("node_off", C.c_void_p), ("xyz", C.c_void_p),
                ("nrm", C.c_void_p), ("wts", C.c_void_p), ("ref_uv", C.c_void_p * (PMAX + 1))]


class TargetsS(C.Structure):
    _fields_ = [("ntarg", C.c_int64), ("xyz", C.c_void_p), ("nrm", C.c_void_p), ("self_node", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("inputs_on_host", C.c_int32), ("ptilde", C.c_int32), ("rho0", C.c_double),
                ("newton_max", C.c_int32), ("eta", C.c_double), ("precision", C.c_int32),
                ("translation", C.c_int32)]


class CSR(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("nnz", C.c_int64), ("npairs", C.c_int64), ("kernel_mask", C.c_uint32),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p * 4)]


class Diag(C.Structure):
    _fields_ = [("npairs", C.c_int64), ("newton_fail", C.c_int64), ("on_edge", C.c_int64), ("u_poor", C.c_int64),
                ("ssq_edges", C.c_int64), ("far_edges", C.c_int64), ("ms_near", C.c_double),
                ("ms_precompute", C.c_double), ("ms_pairs", C.c_double), ("kernel_launches", C.c_int64),
                ("ms_apply_smooth", C.c_double), ("ms_apply_spmv", C.c_double), ("kappa_max", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("nsurf", C.c_int32), ("nrows", C.c_int64), ("nnode", C.c_int64), ("nnz", C.c_int64),
                ("npairs", C.c_int64), ("graph_kernels", C.c_int32), ("tile", C.c_int32 * (PMAX + 1)),
                ("persistent", C.c_int32 * (PMAX + 1)), ("ms_create", C.c_double), ("ms_autotune", C.c_double),
                ("ms_last_execute", C.c_double)]


BATCH_AUTOTUNE = 1
CSR_VIEW = 0x80000000


class RRQError(RuntimeError):
    pass


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load librrq.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise RRQError(f"librrq not found at {path}")
            L = C.CDLL(path)
            L.rrq_status_string.restype = C.c_char_p
            L.rrq_last_error.restype = C.c_char_p
            L.rrq_ctx_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]
            L.rrq_ctx_destroy.argtypes = [C.c_void_p]
            L.rrq_build_corrections.argtypes = [C.c_void_p, C.POINTER(Surface), C.POINTER(TargetsS), C.c_uint32,
                                                C.POINTER(Options), C.POINTER(CSR)]
            L.rrq_csr_copy.argtypes = [C.c_void_p, C.POINTER(CSR), C.c_void_p, C.c_void_p, C.c_void_p * 4, C.c_int32]
            L.rrq_csr_free.argtypes = [C.c_void_p, C.POINTER(CSR)]
            L.rrq_apply.argtypes = [C.c_void_p, C.POINTER(Surface), C.POINTER(TargetsS), C.c_int32, C.POINTER(CSR),
                                    C.c_void_p, C.c_void_p, C.POINTER(Options)]
            L.rrq_apply_correction.argtypes = [C.c_void_p, C.POINTER(CSR), C.c_int32, C.c_void_p, C.c_int64,
                                               C.c_void_p, C.c_int32, C.c_int32]
            L.rrq_last_diagnostics.argtypes = [C.c_void_p, C.POINTER(Diag)]
            L.rrq_measure_fma_peak.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_double)]
            L.rrq_build_corrections_static.argtypes = [C.c_void_p, C.POINTER(Surface), C.POINTER(TargetsS),
                                                       C.c_uint32, C.POINTER(Options), C.c_void_p, C.c_void_p,
                                                       C.c_void_p * 4, C.c_int64, C.POINTER(C.c_int64),
                                                       C.POINTER(C.c_int64)]
            L.rrq_build_corrections_into.argtypes = L.rrq_build_corrections_static.argtypes
            L.rrq_ref_nodes.argtypes = [C.c_int32, C.c_void_p, C.c_void_p]
            L.rrq_batch_create.argtypes = [C.c_void_p, C.c_int32, C.POINTER(Surface), C.POINTER(TargetsS),
                                           C.c_uint32, C.POINTER(Options), C.c_uint32, C.POINTER(C.c_void_p)]
            L.rrq_batch_execute.argtypes = [C.c_void_p, C.c_void_p]
            L.rrq_batch_csr.argtypes = [C.c_void_p, C.c_int32, C.POINTER(CSR), C.c_void_p, C.c_void_p]
            L.rrq_batch_info_get.argtypes = [C.c_void_p, C.POINTER(BatchInfo)]
            L.rrq_batch_destroy.argtypes = [C.c_void_p]
            L.rrq_evaluate_near.argtypes = [C.c_void_p, C.POINTER(Surface), C.POINTER(TargetsS), C.c_uint32,
                                            C.c_void_p, C.c_void_p * 4, C.POINTER(Options)]
            L.rrq_autotune.argtypes = [C.c_void_p, C.POINTER(Surface), C.POINTER(TargetsS), C.c_uint32,
                                       C.POINTER(Options)]
            L.rrq_fit_condition.argtypes = [C.c_void_p, C.POINTER(Surface), C.c_void_p, C.c_int32]
            _lib = L
    return _lib


def ref_nodes(p: int):
    """Reference nodes (n_p, 2) and interpolatory weights (n_p,) of order p (rrq_ref_nodes)."""
    npn = p * (p + 1) // 2
    uv, w = np.zeros((npn, 2)), np.zeros(npn)
    _check(load().rrq_ref_nodes(p, uv.ctypes.data, w.ctypes.data), "rrq_ref_nodes")
    return uv, w


def _check(st: int, what: str):
    if st < 0:
        L = load(False)
        raise RRQError(f"{what}: {L.rrq_status_string(st).decode()} ({L.rrq_last_error().decode()})")
    return st


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _describe(a):
    """(dtype name, element count, contiguous, device) of a torch tensor or numpy array;
    device is ("cuda", index) or ("cpu", None)."""
    if hasattr(a, "data_ptr"):
        dev = (a.device.type, a.device.index if a.device.type == "cuda" else None)
        return str(a.dtype).replace("torch.", ""), int(a.numel()), bool(a.is_contiguous()), dev
    a = np.asarray(a)
    return a.dtype.name, int(a.size), bool(a.flags.c_contiguous), ("cpu", None)


def out_capacity(rowptr, col, vals: dict, kernels, ntarg: int, device: int, host_ok: bool) -> int:
    """Checks the caller's CSR output buffers before any launch and returns the capacity
    in entries: rowptr int64 with at least ntarg + 1 elements, col int32, vals[k] float64
    for every requested kernel k, all contiguous, on cuda:device (or in host memory when
    host_ok).  The capacity is the smallest of col's and every requested vals[k]'s
    length, so the kernels never write past a buffer."""
    def check(name, a, dtype, need=0):
        if a is None:
            raise RRQError(f"{name}: buffer missing")
        dt, n, contig, dev = _describe(a)
        if dt != dtype:
            raise RRQError(f"{name}: dtype {dt}, expected {dtype}")
        if not contig:
            raise RRQError(f"{name}: not contiguous")
        if dev[0] == "cuda" and dev[1] != device:
            raise RRQError(f"{name}: on cuda:{dev[1]}, the context is on cuda:{device}")
        if dev[0] != "cuda" and not host_ok:
            raise RRQError(f"{name}: must be device memory")
        if n < need:
            raise RRQError(f"{name}: {n} elements, at least {need} needed")
        return n
    check("rowptr", rowptr, "int64", ntarg + 1)
    cap = check("col", col, "int32")
    for k in kernels:
        cap = min(cap, check(f"vals[{k}]", vals.get(k), "float64"))
    return cap


class Context:
    """An rrq context bound to a CUDA device and stream (torch stream or raw handle)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RRQError("a CUDA device is required (no CPU fallback)")
        self.L = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self.h = C.c_void_p()
        _check(self.L.rrq_ctx_create(C.byref(self.h), device, C.c_void_p(handle)), "rrq_ctx_create")
        self._keep = []

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.rrq_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- marshalling
    def surface(self, order, node_off, xyz, nrm, wts, ref_uv: dict) -> Surface:
        s = Surface()
        s.npatch = int(order.shape[0])
        s.order, s.node_off, s.xyz, s.nrm, s.wts = (_ptr(a) for a in (order, node_off, xyz, nrm, wts))
        keep = [order, node_off, xyz, nrm, wts]
        for p, uv in ref_uv.items():
            uv = np.ascontiguousarray(uv, dtype=np.float64)
            keep.append(uv)
            s.ref_uv[p] = uv.ctypes.data
        s._keep = keep
        return s

    def targets(self, xyz, nrm, self_node=None) -> TargetsS:
        t = TargetsS()
        t.ntarg = int(xyz.shape[0])
        t.xyz, t.nrm = _ptr(xyz), _ptr(nrm)
        t.self_node = _ptr(self_node)
        t._keep = [xyz, nrm, self_node]
        return t

    # ------------------------------------------------------------- entry points
    def build_corrections(self, surf: Surface, targ: TargetsS, kernels=("S", "D", "SP", "DP"),
                          inputs_on_host: bool = False, rho0: float = 0.0, eta: float = 0.0,
                          newton_max: int = 0, mixed: bool = False, rotation: bool = False) -> CSR:
        """rotation: the O(p^3) rotation-based translation of Step 7 instead of the direct
        sums (rrq_options.translation = 1)."""
        mask = 0
        for k in kernels:
            mask |= KERNEL_BITS[k]
        opt = Options(int(inputs_on_host), 0, rho0, newton_max, eta, int(mixed), int(rotation))
        out = CSR()
        st = self.L.rrq_build_corrections(self.h, C.byref(surf), C.byref(targ), mask, C.byref(opt), C.byref(out))
        _check(st, "rrq_build_corrections")
        self.last_status = st
        return out

    def build_corrections_static(self, surf: Surface, targ: TargetsS, rowptr, col, vals: dict,
                                 kernels=("S", "D", "SP", "DP")):
        """Allocation-free build into caller-owned device buffers (torch CUDA tensors):
        rowptr [ntarg+1] int64, col [capacity] int32, vals {kernel: [capacity] float64}.
        Returns (nnz, npairs)."""
        cap = out_capacity(rowptr, col, vals, kernels, int(targ.ntarg), self.device, host_ok=False)
        mask = 0
        arr = (C.c_void_p * 4)()
        for k in kernels:
            mask |= KERNEL_BITS[k]
            arr[KERNEL_SLOT[k]] = vals[k].data_ptr()
        nnz, npairs = C.c_int64(), C.c_int64()
        opt = Options(0, 0, 0.0, 0, 0.0, 0)
        st = self.L.rrq_build_corrections_static(self.h, C.byref(surf), C.byref(targ), mask, C.byref(opt),
                                                 _ptr(rowptr), _ptr(col), arr, cap, C.byref(nnz), C.byref(npairs))
        _check(st, "rrq_build_corrections_static")
        return nnz.value, npairs.value

    def build_corrections_into(self, surf: Surface, targ: TargetsS, rowptr, col, vals: dict,
                               kernels=("S", "D", "SP", "DP"), inputs_on_host: bool = False,
                               mixed: bool = False, capacity: int = -1, rotation: bool = False):
        """Build into caller-owned buffers the device can address (torch CUDA tensors, or
        page-locked host memory as numpy views of pinned tensors): rowptr [ntarg+1] int64,
        col [capacity] int32, vals {kernel: [capacity] float64}.  The kernels write host
        buffers directly (rrq_build_corrections_into).  Returns (nnz, npairs)."""
        cap = out_capacity(rowptr, col, vals, kernels, int(targ.ntarg), self.device, host_ok=True)
        if capacity >= 0:
            cap = min(cap, capacity)
        mask = 0
        arr = (C.c_void_p * 4)()
        for k in kernels:
            mask |= KERNEL_BITS[k]
            arr[KERNEL_SLOT[k]] = _ptr(vals[k]).value
        nnz, npairs = C.c_int64(), C.c_int64()
        opt = Options(int(inputs_on_host), 0, 0.0, 0, 0.0, int(mixed), int(rotation))
        st = self.L.rrq_build_corrections_into(self.h, C.byref(surf), C.byref(targ), mask, C.byref(opt),
                                               _ptr(rowptr), _ptr(col), arr, cap, C.byref(nnz), C.byref(npairs))
        self.last_nnz = nnz.value
        _check(st, "rrq_build_corrections_into")
        return nnz.value, npairs.value

    def batch(self, surfs, targs, kernels=("S", "D", "SP", "DP"), mixed: bool = False, autotune: bool = False,
              inputs_on_host: bool = False) -> "Batch":
        """Batch plan over several surfaces (rrq_batch_create); see Batch."""
        return Batch(self, surfs, targs, kernels, mixed, autotune, inputs_on_host)

    def evaluate_near(self, surf: Surface, targ: TargetsS, density, outs: dict, inputs_on_host: bool = False):
        """Correction applied to `density` without the matrix (rrq_evaluate_near); outs maps
        kernel names to output arrays [ntarg] (torch CUDA tensors, or numpy with
        inputs_on_host)."""
        mask = 0
        arr = (C.c_void_p * 4)()
        for k, v in outs.items():
            mask |= KERNEL_BITS[k]
            arr[KERNEL_SLOT[k]] = _ptr(v).value
        opt = Options(int(inputs_on_host), 0, 0.0, 0, 0.0, 0)
        st = self.L.rrq_evaluate_near(self.h, C.byref(surf), C.byref(targ), mask, _ptr(density), arr, C.byref(opt))
        _check(st, "rrq_evaluate_near")
        return outs

    def fit_condition(self, surf: Surface, on_host: bool = False):
        """kappa_1(A) of every patch's fit system (rrq_fit_condition): a float64 CUDA tensor
        [npatch], or a numpy array when the surface arrays are host memory."""
        if on_host:
            out = np.empty(surf.npatch)
            ptr = out.ctypes.data
        else:
            import torch
            out = torch.empty(surf.npatch, dtype=torch.float64, device=f"cuda:{self.device}")
            ptr = out.data_ptr()
        _check(self.L.rrq_fit_condition(self.h, C.byref(surf), ptr, int(on_host)), "rrq_fit_condition")
        return out

    def autotune(self, surf: Surface, targ: TargetsS, kernels=("S", "D", "SP", "DP"), mixed: bool = False):
        """Measure the per-pair launch shapes on this problem and keep them in the context
        (rrq_autotune)."""
        mask = 0
        for k in kernels:
            mask |= KERNEL_BITS[k]
        opt = Options(0, 0, 0.0, 0, 0.0, int(mixed))
        _check(self.L.rrq_autotune(self.h, C.byref(surf), C.byref(targ), mask, C.byref(opt)), "rrq_autotune")

    def csr_free(self, csr: CSR):
        _check(self.L.rrq_csr_free(self.h, C.byref(csr)), "rrq_csr_free")

    def csr_to_torch(self, csr: CSR, kernels=("S", "D", "SP", "DP")):
        """Copy a library CSR into torch CUDA tensors: (rowptr, col, {kernel: val})."""
        import torch
        dev = torch.device("cuda", self.device)
        rowptr = torch.empty(csr.nrows + 1, dtype=torch.int64, device=dev)
        col = torch.empty(max(csr.nnz, 1), dtype=torch.int32, device=dev)
        vals = {k: torch.empty(max(csr.nnz, 1), dtype=torch.float64, device=dev) for k in kernels}
        arr = (C.c_void_p * 4)()
        for k, v in vals.items():
            arr[KERNEL_SLOT[k]] = v.data_ptr()
        _check(self.L.rrq_csr_copy(self.h, C.byref(csr), _ptr(rowptr), _ptr(col), arr, 0), "rrq_csr_copy")
        return rowptr, col[: csr.nnz], {k: v[: csr.nnz] for k, v in vals.items()}

    def csr_rows_to_host(self, csr: CSR, rows, kernels=("S", "D", "SP", "DP")):
        """Selected rows of a library CSR as a compact host CSR (rowptr, col, {kernel: val}),
        copied row by row through CSR views (rrq_csr_copy), without copying the matrix."""
        full_rowptr = np.empty(csr.nrows + 1, np.int64)
        _check(self.L.rrq_csr_copy(self.h, C.byref(csr), _ptr(full_rowptr), None, (C.c_void_p * 4)(), 1),
               "rrq_csr_copy")
        rows = np.asarray(rows, np.int64)
        lens = full_rowptr[rows + 1] - full_rowptr[rows]
        rowptr = np.zeros(len(rows) + 1, np.int64)
        np.cumsum(lens, out=rowptr[1:])
        col = np.empty(max(int(rowptr[-1]), 1), np.int32)
        vals = {k: np.empty(max(int(rowptr[-1]), 1), np.float64) for k in kernels}
        for i, t in enumerate(rows):
            v = CSR()
            v.nrows, v.nnz, v.npairs = 1, int(lens[i]), 0
            v.kernel_mask = csr.kernel_mask | CSR_VIEW
            v.rowptr = csr.rowptr + 8 * int(t)
            v.col = csr.col
            for k in range(4):
                v.val[k] = csr.val[k]
            arr = (C.c_void_p * 4)()
            for k, a in vals.items():
                arr[KERNEL_SLOT[k]] = a.ctypes.data + 8 * int(rowptr[i])
            _check(self.L.rrq_csr_copy(self.h, C.byref(v), None, col.ctypes.data + 4 * int(rowptr[i]), arr, 1),
                   "rrq_csr_copy")
        n = int(rowptr[-1])
        return rowptr, col[:n], {k: a[:n] for k, a in vals.items()}

    def csr_to_host(self, csr: CSR, kernels=("S", "D", "SP", "DP"), out=None):
        """Copy a library CSR into (pinned or plain) numpy host buffers."""
        if out is None:
            out = (np.empty(csr.nrows + 1, np.int64), np.empty(max(csr.nnz, 1), np.int32),
                   {k: np.empty(max(csr.nnz, 1), np.float64) for k in kernels})
        rowptr, col, vals = out
        arr = (C.c_void_p * 4)()
        for k, v in vals.items():
            arr[KERNEL_SLOT[k]] = v.ctypes.data
        _check(self.L.rrq_csr_copy(self.h, C.byref(csr), _ptr(rowptr), _ptr(col), arr, 1), "rrq_csr_copy")
        return rowptr, col, vals

    def apply(self, surf: Surface, targ: TargetsS, kernel: str, csr: CSR, density, out,
              inputs_on_host: bool = False, mixed: bool = False):
        opt = Options(int(inputs_on_host), 0, 0.0, 0, 0.0, int(mixed))
        _check(self.L.rrq_apply(self.h, C.byref(surf), C.byref(targ), KERNEL_BITS[kernel],
                                C.byref(csr) if csr is not None else None, _ptr(density), _ptr(out),
                                C.byref(opt)), "rrq_apply")
        return out

    def apply_correction(self, csr: CSR, kernel: str, density, out, accumulate: bool = False,
                         on_host: bool = False):
        """out = (out if accumulate else 0) + C sigma for the correction CSR of `kernel`
        (rrq_apply_correction); density and out are torch CUDA tensors, or numpy arrays
        with on_host."""
        n = int(density.numel()) if hasattr(density, "numel") else int(np.asarray(density).size)
        _check(self.L.rrq_apply_correction(self.h, C.byref(csr), KERNEL_BITS[kernel], _ptr(density), n, _ptr(out),
                                           int(accumulate), int(on_host)), "rrq_apply_correction")
        return out

    def fma_peak_tflops(self, fp32: bool = False) -> float:
        v = C.c_double()
        _check(self.L.rrq_measure_fma_peak(self.h, int(fp32), C.byref(v)), "rrq_measure_fma_peak")
        return v.value

    def diagnostics(self) -> dict:
        d = Diag()
        _check(self.L.rrq_last_diagnostics(self.h, C.byref(d)), "rrq_last_diagnostics")
        return {f: getattr(d, f) for f, _ in Diag._fields_}


def device_inputs(disc, targets, device="cuda"):
    """Torch CUDA copies of a workloads.Discretization and workloads.Targets."""
    import torch
    dev = torch.device(device)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
    return dict(order=t(disc.order, torch.int32), node_off=t(disc.node_off, torch.int64),
                xyz=t(disc.xyz, torch.float64), nrm=t(disc.nrm, torch.float64), wts=t(disc.wts, torch.float64),
                txyz=t(targets.xyz, torch.float64), tnrm=t(targets.nrm, torch.float64),
                tself=t(targets.self_node, torch.int64))


class Batch:
    """Many surfaces built together: rrq_batch_create at construction, execute() launches
    the recorded graph, view(s) is the CSR of surface s (columns local to that surface)."""

    def __init__(self, ctx: Context, surfs, targs, kernels, mixed, autotune, inputs_on_host):
        self.ctx, self.L = ctx, ctx.L
        n = len(surfs)
        if n != len(targs) or n < 1:
            raise RRQError("one targets set per surface is required")
        self._surfs = (Surface * n)(*surfs)
        self._targs = (TargetsS * n)(*targs)
        self._keep = (list(surfs), list(targs))
        mask = 0
        for k in kernels:
            mask |= KERNEL_BITS[k]
        opt = Options(int(inputs_on_host), 0, 0.0, 0, 0.0, int(mixed))
        self.h = C.c_void_p()
        _check(self.L.rrq_batch_create(ctx.h, n, self._surfs, self._targs, mask, C.byref(opt),
                                       BATCH_AUTOTUNE if autotune else 0, C.byref(self.h)), "rrq_batch_create")
        self.nsurf = n
        self.row_start = np.zeros(n + 1, np.int64)
        self.node_start = np.zeros(n + 1, np.int64)
        whole = CSR()
        _check(self.L.rrq_batch_csr(self.h, -1, C.byref(whole), self.row_start.ctypes.data,
                                    self.node_start.ctypes.data), "rrq_batch_csr")
        self.csr = whole

    def execute(self) -> int:
        st = self.L.rrq_batch_execute(self.ctx.h, self.h)
        return _check(st, "rrq_batch_execute")

    def view(self, s: int) -> CSR:
        v = CSR()
        _check(self.L.rrq_batch_csr(self.h, s, C.byref(v), None, None), "rrq_batch_csr")
        return v

    def info(self) -> dict:
        i = BatchInfo()
        _check(self.L.rrq_batch_info_get(self.h, C.byref(i)), "rrq_batch_info_get")
        d = {f: getattr(i, f) for f, _ in BatchInfo._fields_}
        d["tile"] = list(i.tile)
        d["persistent"] = list(i.persistent)
        return d

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.rrq_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
