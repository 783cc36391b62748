"""Host-side checks of the binding that run before any launch (no GPU needed): the CSR
output buffers handed to build_corrections_static / build_corrections_into must have
the right dtypes and lengths, and the capacity passed to the library is the smallest
buffer's length, so that a short values buffer can never be written past its end."""
import ctypes as C

import numpy as np
import pytest

from paper_2411_08342_gb300 import rrq


def _bufs(ntarg=5, ncol=40, nval=40):
    return (np.zeros(ntarg + 1, np.int64), np.zeros(ncol, np.int32),
            {k: np.zeros(nval, np.float64) for k in ("S", "D", "SP", "DP")})


def test_capacity_is_smallest_buffer():
    rp, col, vals = _bufs()
    vals["SP"] = np.zeros(31)
    assert rrq.out_capacity(rp, col, vals, ("S", "D", "SP", "DP"), 5, 0, host_ok=True) == 31
    assert rrq.out_capacity(rp, col, vals, ("S", "D"), 5, 0, host_ok=True) == 40


@pytest.mark.parametrize("bad", ["short_rowptr", "rowptr_int32", "col_int64", "vals_float32", "vals_missing",
                                 "noncontiguous", "host_for_static"])
def test_bad_output_buffers_raise(bad):
    rp, col, vals = _bufs()
    host_ok = True
    if bad == "short_rowptr":
        rp = rp[:5]
    elif bad == "rowptr_int32":
        rp = rp.astype(np.int32)
    elif bad == "col_int64":
        col = col.astype(np.int64)
    elif bad == "vals_float32":
        vals["D"] = vals["D"].astype(np.float32)
    elif bad == "vals_missing":
        del vals["DP"]
    elif bad == "noncontiguous":
        vals["S"] = np.zeros(80)[::2]
    elif bad == "host_for_static":
        host_ok = False
    with pytest.raises(rrq.RRQError):
        rrq.out_capacity(rp, col, vals, ("S", "D", "SP", "DP"), 5, 0, host_ok=host_ok)


class _NoLaunch:
    """Stands in for the loaded library: any call means a launch was attempted."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} was called although the arguments are invalid")


def test_short_values_buffer_raises_before_any_library_call():
    ctx = object.__new__(rrq.Context)
    ctx.L, ctx.h, ctx.device = _NoLaunch(), C.c_void_p(), 0
    targ = rrq.TargetsS()
    targ.ntarg = 5
    rp, col, vals = _bufs()
    vals["D"] = np.zeros(3, np.float32)
    with pytest.raises(rrq.RRQError, match="dtype"):
        ctx.build_corrections_into(None, targ, rp, col, vals)
    with pytest.raises(rrq.RRQError, match="device memory"):
        ctx.build_corrections_static(None, targ, *_bufs())
