"""The C-ABI library builds for sm_103a and exports every function include/rrq.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rrq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rrq_[a-z_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("rrq_build_corrections", "rrq_apply", "rrq_ctx_create", "rrq_csr_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2411_08342_gb300 import build
    lib = ctypes.CDLL(build.build())
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_status_strings_without_gpu():
    from paper_2411_08342_gb300 import rrq
    L = rrq.load()
    assert L.rrq_status_string(0) == b"ok"
    assert L.rrq_status_string(-1) == b"invalid argument"


def test_product_path_does_not_import_oracle():
    """The package never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2411_08342_gb300")
    pat = re.compile(r"(^\s*(from|import)\s+oracle\b)|rrq_oracle|librrq_oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not pat.search(txt), f


def test_ref_nodes_host_function():
    """rrq_ref_nodes (host code, no GPU): the same nodes and interpolatory weights as the
    workload generator for every supported order, exact low-degree moments, and an
    out-of-range order refused."""
    import numpy as np
    import pytest
    from paper_2411_08342_gb300 import rrq, workloads as W
    for p in range(2, rrq.PMAX + 1):
        uv, w = rrq.ref_nodes(p)
        assert np.abs(uv - W.ref_nodes(p)).max() < 1e-15, p
        assert np.abs(w - W.ref_weights(p)).max() < 1e-14, p
        assert abs(w.sum() - 0.5) < 1e-15 and abs(w @ uv[:, 0] - 1 / 6) < 1e-15, p
    with pytest.raises(rrq.RRQError, match="invalid argument"):
        rrq.ref_nodes(rrq.PMAX + 1)
