"""Thin Python binding of libfe (include/fe.h).

Every ``fe_*`` function here has the name and arguments of the C entry point
and only marshals arguments: torch CUDA tensors become device pointers, the
current torch stream becomes the ``stream`` argument, and a non-zero status
raises :class:`FeError`.  All computation happens in the CUDA library; there is
no CPU path.  If ``libfe.so`` has not been built the import fails loudly.

``System`` strings the calls together for one mesh (buffers allocated with
torch) and is what the tests and the benchmark use.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from .build import LIB

FE_OK, FE_ERR_ARG, FE_ERR_OVERFLOW, FE_ERR_CUDA = 0, -1, -2, -3
FE_ERR_BREAKDOWN, FE_ERR_MAXIT, FE_ERR_TIMEOUT, FE_ERR_WORKSPACE = -4, -5, -6, -7
STATUS_NAMES = {0: "FE_OK", -1: "FE_ERR_ARG", -2: "FE_ERR_OVERFLOW", -3: "FE_ERR_CUDA",
                -4: "FE_ERR_BREAKDOWN", -5: "FE_ERR_MAXIT", -6: "FE_ERR_TIMEOUT",
                -7: "FE_ERR_WORKSPACE"}

FE_FMT_CSR, FE_FMT_SELL, FE_FMT_BCRS3, FE_FMT_VBCRS = 0, 1, 2, 3
FORMATS = {"csr": FE_FMT_CSR, "sell": FE_FMT_SELL, "bcrs3": FE_FMT_BCRS3, "vbcrs": FE_FMT_VBCRS}
FE_VAL_F64, FE_VAL_F32, FE_VAL_BF16 = 0, 1, 2
VALUE_TYPES = {"f64": FE_VAL_F64, "f32": FE_VAL_F32, "bf16": FE_VAL_BF16}
TORCH_VALUE = {FE_VAL_F64: torch.float64, FE_VAL_F32: torch.float32, FE_VAL_BF16: torch.bfloat16}
SLICE_ROWS = 32
RESID_WORK_BYTES = 65536 + 64


class FeError(RuntimeError):
    def __init__(self, call: str, status: int):
        self.status = status
        extra = ""
        if status == FE_ERR_CUDA and _lib is not None:
            extra = f" (cuda error {_lib.fe_last_cuda_error()})"
        super().__init__(f"{call} returned {STATUS_NAMES.get(status, status)}{extra}")


class fe_sizes(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_elems", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_faces", ctypes.c_int64), ("n_slices", ctypes.c_int64)]


class fe_matrix(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("value_type", ctypes.c_int32),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("n_slices", ctypes.c_int64), ("n_stored", ctypes.c_int64),
                ("d_row_ptr", ctypes.c_void_p), ("d_slice_ptr", ctypes.c_void_p),
                ("d_cols", ctypes.c_void_p), ("d_vals", ctypes.c_void_p),
                ("d_seg_offsets", ctypes.c_void_p)]


class fe_cg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("relres", ctypes.c_double), ("bnorm", ctypes.c_double)]


class fe_mixed_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("inner_iterations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("relres", ctypes.c_double), ("bnorm", ctypes.c_double)]


BATCH_MAX_SYSTEMS = 256


class fe_batch_plan(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("krhs", ctypes.c_int32),
                ("n_systems", ctypes.c_int32), ("n_chunks", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("max_blocks", ctypes.c_int32),
                ("method", ctypes.c_int32),
                ("d_work", ctypes.c_void_p), ("work_bytes", ctypes.c_size_t),
                ("slot_of", ctypes.c_int32 * BATCH_MAX_SYSTEMS)]


# Exported entry points: name -> (restype, argtypes).  Tests check that the
# shared library exports exactly these names and that include/fe.h declares them.
_VP, _I32, _I64, _D, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "fe_problem_sizes": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(fe_sizes)]),
    "fe_generate_mesh": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
    "fe_assemble_workspace": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_SZ)]),
    "fe_assemble_csr": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP,
                               _VP, _VP, _VP, _SZ, _VP]),
    "fe_sliced_plan": (_I32, [_I32, _I64, _I64, _VP, _VP, _VP, ctypes.POINTER(_I64), _VP]),
    "fe_convert": (_I32, [ctypes.POINTER(fe_matrix), ctypes.POINTER(fe_matrix), _VP]),
    "fe_vbcrs_workspace": (_I32, [_I64, ctypes.POINTER(_SZ)]),
    "fe_vbcrs_plan": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _SZ, ctypes.POINTER(_I64), _VP]),
    "fe_vbcrs_fill": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _VP, _VP]),
    "fe_round_values": (_I32, [_I64, _VP, _I32, _VP, _VP]),
    "fe_spmv": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _VP]),
    "fe_spmv_f32": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _VP]),
    "fe_cg_workspace": (_I32, [ctypes.POINTER(fe_matrix), ctypes.POINTER(_SZ)]),
    "fe_cg_solve": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _D, ctypes.c_int, _D, _VP, _SZ,
                           ctypes.POINTER(fe_cg_result), _VP]),
    "fe_cg_solve_form": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _D, ctypes.c_int, _D,
                                ctypes.c_int, _VP, _SZ, ctypes.POINTER(fe_cg_result), _VP]),
    "fe_cg_sr_workspace": (_I32, [ctypes.POINTER(fe_matrix), ctypes.POINTER(_SZ)]),
    "fe_cg_solve_sr": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _D, ctypes.c_int, _D, _VP, _SZ,
                              ctypes.POINTER(fe_cg_result), _VP]),
    "fe_true_relres": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _VP, _SZ,
                              ctypes.POINTER(_D), _VP]),
    "fe_stencil_spmv": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "fe_stencil_rhs": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "fe_stencil_cg_workspace": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_SZ)]),
    "fe_stencil_cg_solve": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _D, ctypes.c_int,
                                   _D, _VP, _SZ, ctypes.POINTER(fe_cg_result), _VP]),
    "fe_stencil_true_relres": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _SZ,
                                      ctypes.POINTER(_D), _VP]),
    "fe_cg_mixed_workspace": (_I32, [ctypes.POINTER(fe_matrix), ctypes.POINTER(_SZ)]),
    "fe_cg_solve_mixed": (_I32, [ctypes.POINTER(fe_matrix), ctypes.POINTER(fe_matrix), _VP, _VP,
                                 _D, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _D, _VP, _SZ,
                                 ctypes.POINTER(fe_mixed_result), _VP]),
    "fe_cg_solve_noalloc": (_I32, [ctypes.POINTER(fe_matrix), _VP, _VP, _D, ctypes.c_int, _D,
                                   ctypes.POINTER(fe_cg_result), _VP]),
    "fe_cg_batched_workspace": (_I32, [ctypes.c_int, ctypes.POINTER(fe_matrix), ctypes.POINTER(_SZ)]),
    "fe_cg_batched_plan": (_I32, [ctypes.c_int, ctypes.POINTER(fe_matrix), ctypes.POINTER(_VP),
                                  ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _SZ,
                                  ctypes.POINTER(fe_batch_plan), _VP]),
    "fe_cg_batched_launch": (_I32, [ctypes.POINTER(fe_batch_plan), _D, ctypes.c_int, _D, _VP]),
    "fe_cg_batched_results": (_I32, [ctypes.POINTER(fe_batch_plan), ctypes.POINTER(fe_cg_result), _VP]),
    "fe_cg_solve_batched": (_I32, [ctypes.c_int, ctypes.POINTER(fe_matrix), ctypes.POINTER(_VP),
                                   ctypes.POINTER(_VP), _D, ctypes.c_int, ctypes.c_int, _D, _VP, _SZ,
                                   ctypes.POINTER(fe_cg_result), _VP]),
    "fe_nn_conv3d": (_I32, [ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP,
                            ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP]),
    "fe_nn_pack_weights": (_I32, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "fe_nn_mma_image_bytes": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_SZ)]),
    "fe_nn_pack_weights_mma": (_I32, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "fe_nn_conv3d_s1_tc": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP,
                                  ctypes.c_int, ctypes.c_int, _VP]),
    "fe_nn_conv3d_t2_tc": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP]),
    "fe_nn_conv3d_s2_tc": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP]),
    "fe_nn_bf16i_bytes": (_I32, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_SZ)]),
    "fe_nn_to_bf16i": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP]),
    "fe_nn_conv3d_tc_bf16i": (_I32, [ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP]),
    "fe_nn_tc_check": (_I32, [ctypes.POINTER(ctypes.c_int)]),
    "fe_warmstart_blob_layout": (_I32, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "fe_warmstart_workspace": (_I32, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_SZ)]),
    "fe_warmstart_infer": (_I32, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP, _VP, _VP, _SZ,
                                  ctypes.c_int, _VP]),
    "fe_nn_corr_workspace": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                    ctypes.POINTER(_SZ), ctypes.POINTER(ctypes.c_int)]),
    "fe_nn_conv3d_weight_grad": (_I32, [ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _SZ, _VP]),
    "fe_nn_wgrad_tc_workspace": (_I32, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_SZ)]),
    "fe_nn_conv3d_weight_grad_tc": (_I32, [ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP,
                                           ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _SZ, _VP]),
    "fe_nn_channel_sum": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP]),
    "fe_nn_relu_bwd": (_I32, [_VP, _VP, _SZ, _VP]),
    "fe_nn_axpy": (_I32, [ctypes.c_float, _VP, _VP, _SZ, _VP]),
    "fe_nn_head": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP, _VP]),
    "fe_nn_head_bwd": (_I32, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP, _VP, _VP, _VP, _VP,
                              _VP, _SZ, _VP]),
    "fe_nn_mse": (_I32, [_VP, _VP, _VP, _SZ, ctypes.c_float, _VP, _VP, ctypes.c_int, _VP]),
    "fe_nn_adam": (_I32, [_VP, _VP, _VP, _VP, _SZ, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, _VP]),
    "fe_warmstart_input": (_I32, [_VP, _VP, _SZ, _VP, _VP]),
    "fe_warmstart_output": (_I32, [_VP, _VP, _VP, _SZ, _VP, _VP]),
    "fe_inject_barrier_stall": (_I32, [ctypes.c_int]),
    "fe_last_cuda_error": (ctypes.c_int, []),
    "fe_version": (ctypes.c_char_p, []),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"libfe.so is missing ({LIB}); build it with "
                          "`python -m paper_1505_08023_gb300.build` -- there is no CPU fallback")
    lib = ctypes.CDLL(LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(call: str, st: int) -> int:
    if st != FE_OK:
        raise FeError(call, st)
    return st


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------- raw calls

def fe_problem_sizes(nx: int, ny: int, nz: int) -> fe_sizes:
    out = fe_sizes()
    _check("fe_problem_sizes", load().fe_problem_sizes(nx, ny, nz, ctypes.byref(out)))
    return out


def fe_generate_mesh(nx, ny, nz, face_vals, coords, bc_flag, bc_val, conn=None, stream=None):
    return _check("fe_generate_mesh", load().fe_generate_mesh(
        nx, ny, nz, _ptr(face_vals), _ptr(coords), _ptr(bc_flag), _ptr(bc_val), _ptr(conn),
        _stream(stream)))


def fe_assemble_workspace(nx, ny, nz) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_assemble_workspace", load().fe_assemble_workspace(nx, ny, nz, ctypes.byref(n)))
    return n.value


def fe_assemble_csr(nx, ny, nz, coords, bc_flag, bc_val, row_ptr, cols, vals, b, work,
                    stream=None):
    return _check("fe_assemble_csr", load().fe_assemble_csr(
        nx, ny, nz, _ptr(coords), _ptr(bc_flag), _ptr(bc_val), _ptr(row_ptr), _ptr(cols),
        _ptr(vals), _ptr(b), _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def fe_sliced_plan(fmt, n_rows, n_cols, row_ptr, cols, slice_ptr, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check("fe_sliced_plan", load().fe_sliced_plan(
        fmt, n_rows, n_cols, _ptr(row_ptr), _ptr(cols), _ptr(slice_ptr), ctypes.byref(n),
        _stream(stream)))
    return n.value


def fe_vbcrs_workspace(n_rows: int) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_vbcrs_workspace", load().fe_vbcrs_workspace(int(n_rows), ctypes.byref(n)))
    return n.value


def fe_vbcrs_plan(csr: fe_matrix, seg_ptr, work, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check("fe_vbcrs_plan", load().fe_vbcrs_plan(ctypes.byref(csr), _ptr(seg_ptr), _ptr(work),
                                                 work.numel() * work.element_size(), ctypes.byref(n),
                                                 _stream(stream)))
    return n.value


def fe_vbcrs_fill(csr: fe_matrix, seg_ptr, jas, seg_offsets, stream=None):
    return _check("fe_vbcrs_fill", load().fe_vbcrs_fill(ctypes.byref(csr), _ptr(seg_ptr), _ptr(jas),
                                                        _ptr(seg_offsets), _stream(stream)))


def fe_convert(src: fe_matrix, dst: fe_matrix, stream=None):
    return _check("fe_convert", load().fe_convert(ctypes.byref(src), ctypes.byref(dst),
                                                  _stream(stream)))


def fe_round_values(n, src, value_type, dst, stream=None):
    return _check("fe_round_values", load().fe_round_values(n, _ptr(src), value_type, _ptr(dst),
                                                            _stream(stream)))


def fe_spmv(A: fe_matrix, x, y, stream=None):
    return _check("fe_spmv", load().fe_spmv(ctypes.byref(A), _ptr(x), _ptr(y), _stream(stream)))


def fe_spmv_f32(A: fe_matrix, x, y, stream=None):
    return _check("fe_spmv_f32", load().fe_spmv_f32(ctypes.byref(A), _ptr(x), _ptr(y),
                                                    _stream(stream)))


def fe_cg_workspace(A: fe_matrix) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_cg_workspace", load().fe_cg_workspace(ctypes.byref(A), ctypes.byref(n)))
    return n.value


def fe_cg_solve(A: fe_matrix, b, x, tol, maxit, work, timeout_s=0.0, stream=None,
                check=True) -> fe_cg_result:
    res = fe_cg_result()
    st = load().fe_cg_solve(ctypes.byref(A), _ptr(b), _ptr(x), float(tol), int(maxit),
                            float(timeout_s), _ptr(work), work.numel() * work.element_size(),
                            ctypes.byref(res), _stream(stream))
    if check and st not in (FE_OK,):
        raise FeError("fe_cg_solve", st)
    return res


FE_CG_AUTO, FE_CG_THREE_PHASE, FE_CG_TWO_PHASE, FE_CG_RESIDENT = 0, 1, 2, 3


def fe_cg_solve_form(A: fe_matrix, b, x, tol, maxit, form, work, timeout_s=0.0, stream=None,
                     check=True) -> fe_cg_result:
    res = fe_cg_result()
    st = load().fe_cg_solve_form(ctypes.byref(A), _ptr(b), _ptr(x), float(tol), int(maxit),
                                 float(timeout_s), int(form), _ptr(work),
                                 work.numel() * work.element_size(), ctypes.byref(res),
                                 _stream(stream))
    if check and st not in (FE_OK,):
        raise FeError("fe_cg_solve_form", st)
    return res


def fe_cg_sr_workspace(A: fe_matrix) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_cg_sr_workspace", load().fe_cg_sr_workspace(ctypes.byref(A), ctypes.byref(n)))
    return n.value


def fe_cg_solve_sr(A: fe_matrix, b, x, tol, maxit, work, timeout_s=0.0, stream=None,
                   check=True) -> fe_cg_result:
    res = fe_cg_result()
    st = load().fe_cg_solve_sr(ctypes.byref(A), _ptr(b), _ptr(x), float(tol), int(maxit),
                               float(timeout_s), _ptr(work), work.numel() * work.element_size(),
                               ctypes.byref(res), _stream(stream))
    if check and st not in (FE_OK,):
        raise FeError("fe_cg_solve_sr", st)
    return res


def fe_cg_mixed_workspace(A_lo: fe_matrix) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_cg_mixed_workspace", load().fe_cg_mixed_workspace(ctypes.byref(A_lo), ctypes.byref(n)))
    return n.value


FE_MIXED_RELIABLE, FE_MIXED_RESTART = 0, 1


def fe_cg_solve_mixed(A64: fe_matrix, A_lo: fe_matrix, b, x, tol, mode, max_outer, inner_tol,
                      max_inner, work, timeout_s=0.0, stream=None, check=True) -> fe_mixed_result:
    res = fe_mixed_result()
    st = load().fe_cg_solve_mixed(ctypes.byref(A64), ctypes.byref(A_lo), _ptr(b), _ptr(x),
                                  float(tol), int(mode), int(max_outer), float(inner_tol),
                                  int(max_inner),
                                  float(timeout_s), _ptr(work), work.numel() * work.element_size(),
                                  ctypes.byref(res), _stream(stream))
    if check and st != FE_OK:
        raise FeError("fe_cg_solve_mixed", st)
    return res


NOALLOC_MAX_ROWS = 262144


def fe_cg_solve_noalloc(A: fe_matrix, b, x, tol, maxit, timeout_s=0.0, stream=None,
                        check=True) -> fe_cg_result:
    """fe_cg_solve with the library's built-in scratch (no workspace argument)."""
    res = fe_cg_result()
    st = load().fe_cg_solve_noalloc(ctypes.byref(A), _ptr(b), _ptr(x), float(tol), int(maxit),
                                    float(timeout_s), ctypes.byref(res), _stream(stream))
    if check and st != FE_OK:
        raise FeError("fe_cg_solve_noalloc", st)
    return res


def fe_true_relres(A: fe_matrix, b, x, work, stream=None) -> float:
    out = ctypes.c_double(0.0)
    _check("fe_true_relres", load().fe_true_relres(
        ctypes.byref(A), _ptr(b), _ptr(x), _ptr(work), work.numel() * work.element_size(),
        ctypes.byref(out), _stream(stream)))
    return out.value


# ---------------------------------------------------------------- matrix-free form

def fe_stencil_spmv(nx, ny, nz, x, y, stream=None):
    return _check("fe_stencil_spmv", load().fe_stencil_spmv(nx, ny, nz, _ptr(x), _ptr(y), _stream(stream)))


def fe_stencil_rhs(nx, ny, nz, bc_val, b, stream=None):
    return _check("fe_stencil_rhs", load().fe_stencil_rhs(nx, ny, nz, _ptr(bc_val), _ptr(b), _stream(stream)))


def fe_stencil_cg_workspace(nx, ny, nz) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_stencil_cg_workspace", load().fe_stencil_cg_workspace(nx, ny, nz, ctypes.byref(n)))
    return n.value


def fe_stencil_cg_solve(nx, ny, nz, b, x, tol, maxit, work, timeout_s=0.0, stream=None,
                        check=True) -> fe_cg_result:
    res = fe_cg_result()
    st = load().fe_stencil_cg_solve(nx, ny, nz, _ptr(b), _ptr(x), float(tol), int(maxit), float(timeout_s),
                                    _ptr(work), work.numel() * work.element_size(), ctypes.byref(res),
                                    _stream(stream))
    if check and st != FE_OK:
        raise FeError("fe_stencil_cg_solve", st)
    return res


def fe_stencil_true_relres(nx, ny, nz, b, x, work, stream=None) -> float:
    out = ctypes.c_double(0.0)
    _check("fe_stencil_true_relres", load().fe_stencil_true_relres(
        nx, ny, nz, _ptr(b), _ptr(x), _ptr(work), work.numel() * work.element_size(), ctypes.byref(out),
        _stream(stream)))
    return out.value


class StencilSystem:
    """Matrix-free form of one nx x ny x nz problem: the mesh's boundary data,
    the right-hand side and the CG workspace (no matrix, no coordinates)."""

    def __init__(self, nx: int, ny: int | None = None, nz: int | None = None, device="cuda",
                 face_vals: torch.Tensor | None = None):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        self.dims = (nx, ny, nz)
        self.device = torch.device(device)
        self.m = (nx + 1) * (ny + 1) * (nz + 1)
        self.bc_flag = torch.empty(self.m, dtype=torch.uint8, device=self.device)
        self.bc_val = torch.empty(self.m, dtype=torch.float64, device=self.device)
        self.b = torch.empty(self.m, dtype=torch.float64, device=self.device)
        self.face_vals = face_vals
        self.work = _alloc_bytes(fe_stencil_cg_workspace(*self.dims), self.device)

    def build(self, stream=None):
        fe_generate_mesh(*self.dims, self.face_vals, None, self.bc_flag, self.bc_val, None, stream)
        fe_stencil_rhs(*self.dims, self.bc_val, self.b, stream)
        return self

    def spmv(self, x, y, stream=None):
        fe_stencil_spmv(*self.dims, x, y, stream)

    def solve(self, x, tol=1e-10, maxit=100000, timeout_s=0.0, stream=None, check=True) -> fe_cg_result:
        return fe_stencil_cg_solve(*self.dims, self.b, x, tol, maxit, self.work, timeout_s, stream, check)

    def true_relres(self, x, stream=None) -> float:
        return fe_stencil_true_relres(*self.dims, self.b, x, self.work, stream)


def fe_inject_barrier_stall(barrier_index: int):
    return _check("fe_inject_barrier_stall", load().fe_inject_barrier_stall(barrier_index))


def _descs(mats) -> ctypes.Array:
    arr = (fe_matrix * len(mats))()
    for i, d in enumerate(mats):
        arr[i] = d
    return arr


def _ptrs(tensors) -> ctypes.Array:
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _ptr(t)
    return arr


def fe_cg_batched_workspace(mats) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_cg_batched_workspace",
           load().fe_cg_batched_workspace(len(mats), _descs(mats), ctypes.byref(n)))
    return n.value


BATCH_TEXTBOOK, BATCH_SINGLE_REDUCTION = 0, 1


def fe_cg_batched_plan(mats, bs, xs, krhs, work, blocks_per_sm=0, stream=None,
                       method=BATCH_TEXTBOOK) -> fe_batch_plan:
    plan = fe_batch_plan()
    _check("fe_cg_batched_plan", load().fe_cg_batched_plan(
        len(mats), _descs(mats), _ptrs(bs), _ptrs(xs), int(krhs), int(method), int(blocks_per_sm),
        _ptr(work),
        work.numel() * work.element_size(), ctypes.byref(plan), _stream(stream)))
    return plan


def fe_cg_batched_launch(plan: fe_batch_plan, tol, maxit, timeout_s=0.0, stream=None):
    return _check("fe_cg_batched_launch", load().fe_cg_batched_launch(
        ctypes.byref(plan), float(tol), int(maxit), float(timeout_s), _stream(stream)))


def fe_cg_batched_results(plan: fe_batch_plan, stream=None):
    n = plan.n_systems
    res = (fe_cg_result * n)()
    st = load().fe_cg_batched_results(ctypes.byref(plan), res, _stream(stream))
    return st, [res[i] for i in range(n)]


def fe_cg_solve_batched(mats, bs, xs, tol, maxit, krhs, work, timeout_s=0.0, stream=None):
    n = len(mats)
    res = (fe_cg_result * n)()
    st = load().fe_cg_solve_batched(n, _descs(mats), _ptrs(bs), _ptrs(xs), float(tol), int(maxit),
                                    int(krhs), float(timeout_s), _ptr(work),
                                    work.numel() * work.element_size(), res, _stream(stream))
    return st, [res[i] for i in range(n)]


FE_NN_S1, FE_NN_S2, FE_NN_T2 = 0, 1, 2
NN_MODES = {"s1": FE_NN_S1, "s2": FE_NN_S2, "t2": FE_NN_T2}


def _dims(d):
    return (ctypes.c_int * 3)(*[int(v) for v in d])


def fe_nn_conv3d(mode, x, cin, dims_in, w_bf16, bias, y, cout, dims_out, relu, stream=None):
    return _check("fe_nn_conv3d", load().fe_nn_conv3d(
        int(mode), _ptr(x), int(cin), _dims(dims_in), _ptr(w_bf16), _ptr(bias), _ptr(y), int(cout),
        _dims(dims_out), int(relu), _stream(stream)))


TC_COUT = (16, 32, 64)


def fe_nn_mma_image_bytes(cin, cout) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_nn_mma_image_bytes", load().fe_nn_mma_image_bytes(int(cin), int(cout), ctypes.byref(n)))
    return n.value


def fe_nn_pack_weights_mma(w_bf16, cin, cout, img, stream=None):
    return _check("fe_nn_pack_weights_mma", load().fe_nn_pack_weights_mma(
        _ptr(w_bf16), int(cin), int(cout), _ptr(img), _stream(stream)))


def fe_nn_conv3d_s1_tc(x, cin, dims, img, bias, y, cout, relu, stream=None):
    return _check("fe_nn_conv3d_s1_tc", load().fe_nn_conv3d_s1_tc(
        _ptr(x), int(cin), _dims(dims), _ptr(img), _ptr(bias), _ptr(y), int(cout), int(relu),
        _stream(stream)))


def fe_nn_conv3d_t2_tc(x, cin, dims_in, img, bias, y, cout, dims_out, relu, stream=None):
    return _check("fe_nn_conv3d_t2_tc", load().fe_nn_conv3d_t2_tc(
        _ptr(x), int(cin), _dims(dims_in), _ptr(img), _ptr(bias), _ptr(y), int(cout), _dims(dims_out),
        int(relu), _stream(stream)))


def fe_nn_conv3d_s2_tc(x, cin, dims_in, img, bias, y, cout, dims_out, relu, stream=None):
    return _check("fe_nn_conv3d_s2_tc", load().fe_nn_conv3d_s2_tc(
        _ptr(x), int(cin), _dims(dims_in), _ptr(img), _ptr(bias), _ptr(y), int(cout), _dims(dims_out),
        int(relu), _stream(stream)))


def conv3d_tc(mode, x, cin, dims_in, img, bias, y, cout, dims_out, relu, stream=None):
    """The tensor-core convolution of `mode` ("s1", "s2" or "t2")."""
    if mode == "s1":
        return fe_nn_conv3d_s1_tc(x, cin, dims_in, img, bias, y, cout, relu, stream)
    if mode == "s2":
        return fe_nn_conv3d_s2_tc(x, cin, dims_in, img, bias, y, cout, dims_out, relu, stream)
    return fe_nn_conv3d_t2_tc(x, cin, dims_in, img, bias, y, cout, dims_out, relu, stream)


def fe_nn_bf16i_bytes(c, dims) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_nn_bf16i_bytes", load().fe_nn_bf16i_bytes(int(c), _dims(dims), ctypes.byref(n)))
    return n.value


def fe_nn_to_bf16i(x, c, dims, out, stream=None):
    return _check("fe_nn_to_bf16i", load().fe_nn_to_bf16i(_ptr(x), int(c), _dims(dims), _ptr(out),
                                                          _stream(stream)))


def fe_nn_conv3d_tc_bf16i(mode, x16, cin, dims_in, img, bias, y, cout, dims_out, relu, stream=None):
    m = NN_MODES[mode] if isinstance(mode, str) else int(mode)
    return _check("fe_nn_conv3d_tc_bf16i", load().fe_nn_conv3d_tc_bf16i(
        m, _ptr(x16), int(cin), _dims(dims_in), _ptr(img), _ptr(bias), _ptr(y), int(cout), _dims(dims_out),
        int(relu), _stream(stream)))


def bf16i_buffer(c, dims, device="cuda") -> torch.Tensor:
    """Buffer for a BF16 8-channel-interleaved volume."""
    return _alloc_bytes(fe_nn_bf16i_bytes(c, dims), device)


def fe_nn_tc_check() -> int:
    f = ctypes.c_int(0)
    _check("fe_nn_tc_check", load().fe_nn_tc_check(ctypes.byref(f)))
    return f.value


def fe_warmstart_blob_layout(channels):
    """(offsets of the 28 sections, total bytes) of a warm-start weight blob."""
    ch = (ctypes.c_int * 4)(*[int(c) for c in channels])
    offs = (ctypes.c_size_t * 28)()
    n = ctypes.c_size_t(0)
    _check("fe_warmstart_blob_layout", load().fe_warmstart_blob_layout(ch, offs, ctypes.byref(n)))
    return [offs[i] for i in range(28)], n.value


def fe_warmstart_workspace(n_nodes, channels) -> int:
    ch = (ctypes.c_int * 4)(*[int(c) for c in channels])
    n = ctypes.c_size_t(0)
    _check("fe_warmstart_workspace", load().fe_warmstart_workspace(int(n_nodes), ch, ctypes.byref(n)))
    return n.value


def fe_warmstart_infer(n_nodes, channels, blob, bc_flag, bc_val, x0, work, tensor_cores=True, stream=None):
    ch = (ctypes.c_int * 4)(*[int(c) for c in channels])
    return _check("fe_warmstart_infer", load().fe_warmstart_infer(
        int(n_nodes), ch, _ptr(blob), _ptr(bc_flag), _ptr(bc_val), _ptr(x0), _ptr(work),
        work.numel() * work.element_size(), int(bool(tensor_cores)), _stream(stream)))


def mma_image(cin, cout, device="cuda") -> torch.Tensor:
    """Buffer for a tensor-core weight image (16-byte aligned)."""
    return _alloc_bytes(fe_nn_mma_image_bytes(cin, cout), device)


def fe_nn_pack_weights(w, cin, cout, transpose, flip, out, stream=None):
    return _check("fe_nn_pack_weights", load().fe_nn_pack_weights(
        _ptr(w), int(cin), int(cout), int(transpose), int(flip), _ptr(out), _stream(stream)))


def fe_nn_corr_workspace(stride, ca, dims_a, cb):
    n = ctypes.c_size_t(0)
    k = ctypes.c_int(0)
    _check("fe_nn_corr_workspace", load().fe_nn_corr_workspace(
        int(stride), int(ca), _dims(dims_a), int(cb), ctypes.byref(n), ctypes.byref(k)))
    return n.value, k.value


def fe_nn_conv3d_weight_grad(mode, x, cin, dims_in, dy, cout, dims_out, dw, work, stream=None):
    return _check("fe_nn_conv3d_weight_grad", load().fe_nn_conv3d_weight_grad(
        int(mode), _ptr(x), int(cin), _dims(dims_in), _ptr(dy), int(cout), _dims(dims_out), _ptr(dw),
        _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def fe_nn_wgrad_tc_workspace(mode, cin, dims_in, cout, dims_out) -> int:
    n = ctypes.c_size_t(0)
    _check("fe_nn_wgrad_tc_workspace", load().fe_nn_wgrad_tc_workspace(
        int(mode), int(cin), _dims(dims_in), int(cout), _dims(dims_out), ctypes.byref(n)))
    return n.value


def fe_nn_conv3d_weight_grad_tc(mode, x, cin, dims_in, dy, cout, dims_out, dw, work, stream=None):
    return _check("fe_nn_conv3d_weight_grad_tc", load().fe_nn_conv3d_weight_grad_tc(
        int(mode), _ptr(x), int(cin), _dims(dims_in), _ptr(dy), int(cout), _dims(dims_out), _ptr(dw),
        _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def fe_nn_channel_sum(dy, c, dims, db, stream=None):
    return _check("fe_nn_channel_sum", load().fe_nn_channel_sum(_ptr(dy), int(c), _dims(dims), _ptr(db),
                                                                _stream(stream)))


def fe_nn_relu_bwd(y, dy, stream=None):
    return _check("fe_nn_relu_bwd", load().fe_nn_relu_bwd(_ptr(y), _ptr(dy), dy.numel(), _stream(stream)))


def fe_nn_axpy(a, x, y, stream=None):
    return _check("fe_nn_axpy", load().fe_nn_axpy(float(a), _ptr(x), _ptr(y), y.numel(), _stream(stream)))


def fe_nn_head(h, c, dims, w_bf16, b, out, stream=None):
    return _check("fe_nn_head", load().fe_nn_head(_ptr(h), int(c), _dims(dims), _ptr(w_bf16), _ptr(b),
                                                  _ptr(out), _stream(stream)))


def fe_nn_head_bwd(h, c, dims, w_bf16, dout, dh, dw, db, work, stream=None):
    return _check("fe_nn_head_bwd", load().fe_nn_head_bwd(
        _ptr(h), int(c), _dims(dims), _ptr(w_bf16), _ptr(dout), _ptr(dh), _ptr(dw), _ptr(db), _ptr(work),
        work.numel() * work.element_size(), _stream(stream)))


def fe_nn_mse(pred, target, bc_flag, scale, dpred, parts, stream=None):
    return _check("fe_nn_mse", load().fe_nn_mse(
        _ptr(pred), _ptr(target), _ptr(bc_flag), pred.numel(), float(scale), _ptr(dpred), _ptr(parts),
        parts.numel(), _stream(stream)))


def fe_nn_adam(w, g, m, v, lr_t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    return _check("fe_nn_adam", load().fe_nn_adam(_ptr(w), _ptr(g), _ptr(m), _ptr(v), w.numel(),
                                                  float(lr_t), float(beta1), float(beta2), float(eps),
                                                  _stream(stream)))


def fe_warmstart_input(bc_flag, bc_val, x, stream=None):
    return _check("fe_warmstart_input", load().fe_warmstart_input(
        _ptr(bc_flag), _ptr(bc_val), bc_flag.numel(), _ptr(x), _stream(stream)))


def fe_warmstart_output(pred, bc_flag, bc_val, x0, stream=None):
    return _check("fe_warmstart_output", load().fe_warmstart_output(
        _ptr(pred), _ptr(bc_flag), _ptr(bc_val), bc_flag.numel(), _ptr(x0), _stream(stream)))


def fe_version() -> str:
    return load().fe_version().decode()


# ---------------------------------------------------------------- one mesh, end to end

def _alloc_bytes(n: int, device) -> torch.Tensor:
    # 256-byte alignment comes with the caching allocator (512-byte blocks)
    return torch.empty(max(n, 1), dtype=torch.uint8, device=device)


@dataclass
class DeviceMatrix:
    """A matrix in one format plus the tensors that own its memory."""
    desc: fe_matrix
    tensors: dict

    @property
    def format(self) -> int:
        return self.desc.format

    def stored_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.tensors.values())


class System:
    """Mesh, assembled CSR system and solver buffers for one nx x ny x nz problem."""

    def __init__(self, nx: int, ny: int | None = None, nz: int | None = None, device="cuda",
                 face_vals: torch.Tensor | None = None, keep_conn: bool = False):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        self.dims = (nx, ny, nz)
        self.device = torch.device(device)
        self.sizes = fe_problem_sizes(nx, ny, nz)
        m, nnz = self.sizes.n_rows, self.sizes.nnz
        dev = self.device
        self.coords = torch.empty((m, 3), dtype=torch.float64, device=dev)
        self.bc_flag = torch.empty(m, dtype=torch.uint8, device=dev)
        self.bc_val = torch.empty(m, dtype=torch.float64, device=dev)
        self.conn = (torch.empty((self.sizes.n_elems, 8), dtype=torch.int32, device=dev)
                     if keep_conn else None)
        self.row_ptr = torch.empty(m + 1, dtype=torch.int32, device=dev)
        self.cols = torch.empty(nnz, dtype=torch.int32, device=dev)
        self.vals = torch.empty(nnz, dtype=torch.float64, device=dev)
        self.b = torch.empty(m, dtype=torch.float64, device=dev)
        self.face_vals = face_vals
        self._asm_work = None
        self._formats: dict = {}

    # -- pipeline steps
    def generate_mesh(self, stream=None):
        fe_generate_mesh(*self.dims, self.face_vals, self.coords, self.bc_flag, self.bc_val,
                         self.conn, stream)

    def assemble(self, stream=None, keep_workspace: bool = False):
        if self._asm_work is None:
            self._asm_work = _alloc_bytes(fe_assemble_workspace(*self.dims), self.device)
        fe_assemble_csr(*self.dims, self.coords, self.bc_flag, self.bc_val, self.row_ptr,
                        self.cols, self.vals, self.b, self._asm_work, stream)
        if not keep_workspace:
            # the caching allocator reuses the block only after work already
            # queued on the stream that used it
            if stream is not None:
                self._asm_work.record_stream(stream)
            self._asm_work = None

    def build(self, stream=None):
        self.generate_mesh(stream)
        self.assemble(stream)
        return self

    @property
    def m(self) -> int:
        return self.sizes.n_rows

    def csr(self) -> DeviceMatrix:
        d = fe_matrix(FE_FMT_CSR, FE_VAL_F64, self.m, self.m, self.sizes.n_slices,
                      self.sizes.nnz, self.row_ptr.data_ptr(), None, self.cols.data_ptr(),
                      self.vals.data_ptr())
        return DeviceMatrix(d, {"row_ptr": self.row_ptr, "cols": self.cols, "vals": self.vals})

    def matrix(self, fmt: str = "csr", value: str = "f64", stream=None) -> DeviceMatrix:
        """The assembled matrix in a storage format (converted and cached on first use)."""
        key = (fmt, value)
        if key in self._formats:
            return self._formats[key]
        f, vt = FORMATS[fmt], VALUE_TYPES[value]
        src = self.csr()
        if f == FE_FMT_CSR:
            if vt == FE_VAL_F64:
                return src
            v = torch.empty(self.sizes.nnz, dtype=TORCH_VALUE[vt], device=self.device)
            fe_round_values(self.sizes.nnz, self.vals, vt, v, stream)
            d = fe_matrix(f, vt, self.m, self.m, self.sizes.n_slices, self.sizes.nnz,
                          self.row_ptr.data_ptr(), None, self.cols.data_ptr(), v.data_ptr())
            dm = DeviceMatrix(d, {"row_ptr": self.row_ptr, "cols": self.cols, "vals": v})
        elif f == FE_FMT_VBCRS:
            # the paper's BCRS: segment arrays over the CSR values (or a rounded copy)
            v = self.vals
            if vt != FE_VAL_F64:
                v = torch.empty(self.sizes.nnz, dtype=TORCH_VALUE[vt], device=self.device)
                fe_round_values(self.sizes.nnz, self.vals, vt, v, stream)
            seg_ptr = torch.empty(self.m + 1, dtype=torch.int32, device=self.device)
            work = _alloc_bytes(fe_vbcrs_workspace(self.m), self.device)
            nns = fe_vbcrs_plan(src.desc, seg_ptr, work, stream)
            jas = torch.empty(nns, dtype=torch.int32, device=self.device)
            offs = torch.empty(nns + 1, dtype=torch.int32, device=self.device)
            fe_vbcrs_fill(src.desc, seg_ptr, jas, offs, stream)
            d = fe_matrix(f, vt, self.m, self.m, self.sizes.n_slices, nns, seg_ptr.data_ptr(), None,
                          jas.data_ptr(), v.data_ptr(), offs.data_ptr())
            dm = DeviceMatrix(d, {"seg_ptr": seg_ptr, "jas": jas, "seg_offsets": offs, "vals": v})
        else:
            ns = self.sizes.n_slices
            sp = torch.empty(ns + 1, dtype=torch.int64, device=self.device)
            n_stored = fe_sliced_plan(f, self.m, self.m, self.row_ptr, self.cols, sp, stream)
            cols = torch.empty(n_stored, dtype=torch.int32, device=self.device)
            nv = n_stored * (3 if f == FE_FMT_BCRS3 else 1)
            v = torch.empty(nv, dtype=TORCH_VALUE[vt], device=self.device)
            d = fe_matrix(f, vt, self.m, self.m, ns, n_stored, None, sp.data_ptr(),
                          cols.data_ptr(), v.data_ptr())
            fe_convert(src.desc, d, stream)
            dm = DeviceMatrix(d, {"slice_ptr": sp, "cols": cols, "vals": v})
        self._formats[key] = dm
        return dm

    def convert(self, fmt: str = "bcrs3", value: str = "f64", stream=None) -> DeviceMatrix:
        """Rebuild the copy in `fmt` from the current CSR values, reusing its
        buffers when the layout size is unchanged (the conversion the solver
        runs at the start of every solve)."""
        key = (fmt, value)
        dm = self._formats.get(key)
        f, vt = FORMATS[fmt], VALUE_TYPES[value]
        if dm is None or f in (FE_FMT_CSR, FE_FMT_VBCRS):
            self._formats.pop(key, None)
            return self.matrix(fmt, value, stream)
        sp = dm.tensors["slice_ptr"]
        n_stored = fe_sliced_plan(f, self.m, self.m, self.row_ptr, self.cols, sp, stream)
        if n_stored != dm.desc.n_stored:
            self._formats.pop(key, None)
            return self.matrix(fmt, value, stream)
        fe_convert(self.csr().desc, dm.desc, stream)
        return dm

    def drop_formats(self):
        self._formats.clear()


def cg_workspace(A: DeviceMatrix, device="cuda") -> torch.Tensor:
    return _alloc_bytes(fe_cg_workspace(A.desc), device)


def sr_workspace(A: DeviceMatrix, device="cuda") -> torch.Tensor:
    return _alloc_bytes(fe_cg_sr_workspace(A.desc), device)


def mixed_workspace(A_lo: DeviceMatrix, device="cuda") -> torch.Tensor:
    return _alloc_bytes(fe_cg_mixed_workspace(A_lo.desc), device)


def resid_workspace(device="cuda") -> torch.Tensor:
    return _alloc_bytes(RESID_WORK_BYTES, device)


class Batch:
    """Independent problems of different mesh sizes and boundary data, ready
    for the batched solve.  Problems with equal mesh share one matrix (the
    assembled matrix does not depend on the boundary values); each keeps its
    own right-hand side and solution vector."""

    def __init__(self, sizes, faces=None, fmt: str = "bcrs3", device="cuda"):
        self.sizes = [int(n) for n in sizes]
        self.fmt = fmt
        self.device = torch.device(device)
        self.reps = {}       # mesh size -> System holding the shared matrix
        self.b, self.x = [], []
        for i, n in enumerate(self.sizes):
            fv = None
            if faces is not None and faces[i] is not None:
                fv = torch.as_tensor(faces[i], dtype=torch.float64, device=self.device)
            s = System(n, device=self.device, face_vals=fv).build()
            self.b.append(s.b)
            self.x.append(torch.zeros(s.m, dtype=torch.float64, device=self.device))
            if n not in self.reps:
                self.reps[n] = s
                s.matrix(fmt, "f64")
            else:
                del s
        self.mats = [self.reps[n].matrix(fmt, "f64").desc for n in self.sizes]

    def mats_for(self, fmt: str):
        """Descriptors of the shared matrices in another storage format."""
        return [self.reps[n].matrix(fmt, "f64").desc for n in self.sizes]

    def reset(self):
        for x in self.x:
            x.zero_()

    def workspace(self) -> torch.Tensor:
        return _alloc_bytes(fe_cg_batched_workspace(self.mats), self.device)
