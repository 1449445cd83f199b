"""The C-ABI library loads on a host without a GPU, exports every entry point
that include/fe.h declares (and nothing else under the fe_ prefix), and
checks its arguments before touching the device.  No compute call is made.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1505_08023_gb300.fe as fe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "fe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", text))


def exported_functions():
    out = subprocess.run(["nm", "-D", "--defined-only", fe.LIB], capture_output=True, text=True,
                         check=True).stdout
    return {line.split()[-1] for line in out.splitlines() if re.search(r" T fe_", line)}


def test_library_exports_header():
    fe.load()
    declared = header_functions()
    assert declared == set(fe.SIGNATURES), declared ^ set(fe.SIGNATURES)
    assert exported_functions() == declared


def test_sizes_closed_form():
    for dims in [(1, 1, 1), (30, 30, 30), (256, 256, 256), (400, 400, 400), (3, 7, 5)]:
        s = fe.fe_problem_sizes(*dims)
        nx, ny, nz = dims
        assert s.n_rows == (nx + 1) * (ny + 1) * (nz + 1)
        assert s.nnz == (3 * nx + 1) * (3 * ny + 1) * (3 * nz + 1)
        assert s.n_elems == nx * ny * nz
        assert s.n_slices == -(-s.n_rows // 32)
    # the int32 row pointer overflows at 430 elements per axis
    assert fe.fe_problem_sizes(429, 429, 429).nnz < 2 ** 31
    with pytest.raises(fe.FeError) as e:
        fe.fe_problem_sizes(430, 430, 430)
    assert e.value.status == fe.FE_ERR_OVERFLOW
    with pytest.raises(fe.FeError) as e:
        fe.fe_problem_sizes(0, 4, 4)
    assert e.value.status == fe.FE_ERR_ARG


def test_argument_checks_precede_device_work():
    lib = fe.load()
    # NULL output arrays are rejected before anything is enqueued
    assert lib.fe_generate_mesh(4, 4, 4, None, None, None, None, None, None) == fe.FE_ERR_ARG
    assert lib.fe_assemble_csr(4, 4, 4, None, None, None, None, None, None, None, None, 0,
                               None) == fe.FE_ERR_ARG
    n = ctypes.c_size_t(0)
    assert lib.fe_assemble_workspace(4, 5, 6, ctypes.byref(n)) == fe.FE_OK
    assert n.value == 4 * 5 * 6 * 36 * 8
    bad = fe.fe_matrix(7, 0, 10, 10, 1, 10, None, None, None, None)
    assert lib.fe_spmv(ctypes.byref(bad), None, None, None) == fe.FE_ERR_ARG
    assert lib.fe_cg_workspace(ctypes.byref(bad), ctypes.byref(n)) == fe.FE_ERR_ARG
    assert lib.fe_inject_barrier_stall(-2) == fe.FE_ERR_ARG
    assert lib.fe_inject_barrier_stall(-1) == fe.FE_OK
    # workspace query of a well-formed descriptor needs no device
    ok = fe.fe_matrix(fe.FE_FMT_CSR, fe.FE_VAL_F64, 100, 100, 4, 500, 8, None, 8, 8)
    assert lib.fe_cg_workspace(ctypes.byref(ok), ctypes.byref(n)) == fe.FE_OK
    assert n.value >= 3 * 128 * 8


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import importlib
    monkeypatch.setattr(fe, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fe, "_lib", None)
    with pytest.raises(ImportError):
        fe.load()
