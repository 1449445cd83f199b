"""Mixed-precision form (FP32 or BF16 matrix values, FP32 inner CG with FP32
accumulation, FP64 residual, refinement and global dot products) judged
against the FP64 oracle, through the C ABI.

Criteria (the FP64 path's, see test_gpu_cg.py): the oracle's true relative
residual of the result <= 1.5e-10, and the result at least as accurate as the
oracle's own FP64 CG solution at 1e-10: ||x - x*|| <= 2 ||x_oracle - x*|| +
1e-12 ||x*||, x* the oracle solved to 1e-14.
"""
import numpy as np
import pytest
import torch

import fe_inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_1505_08023_gb300.fe as fe_mod
    fe_mod.load()
    return fe_mod


REF = {}


def reference(dims, face=None):
    key = (dims, None if face is None else face.tobytes())
    if key not in REF:
        sysm = oracle.build_system(*dims, face)
        x, it, rel, st = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                   tol=1e-10, maxit=5000)
        xs, _, _, _ = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                tol=1e-14, maxit=20000)
        REF[key] = (sysm, x, xs)
    return REF[key]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


INNER_TOL = {"f32": 1e-5, "bf16": 1e-3}


def solve_mixed(fe, s, fmt, value, tol=1e-10, inner_tol=None, max_outer=30):
    A64 = s.matrix("csr", "f64")
    Alo = s.matrix(fmt, value)
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    work = fe.mixed_workspace(Alo)
    res = fe.fe_cg_solve_mixed(A64.desc, Alo.desc, s.b, x, tol, max_outer,
                               inner_tol or INNER_TOL[value], 5000, work, check=False)
    return x, res


@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("value", ["f32", "bf16"])
def test_mixed_matches_fp64_oracle(fe, fmt, value):
    dims = (30, 30, 30)
    sysm, x_or, x_star = reference(dims)
    s = fe.System(*dims).build()
    x, res = solve_mixed(fe, s, fmt, value)
    assert res.status == fe.FE_OK and res.relres <= 1e-10
    xg = x.cpu().numpy()
    tr = oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg)
    assert tr <= 1.5e-10
    assert rel(xg, x_star) <= 2.0 * rel(x_or, x_star) + 1e-12
    assert res.outer_iterations >= 1 and res.inner_iterations >= res.outer_iterations


@pytest.mark.parametrize("value", ["f32", "bf16"])
def test_mixed_face_data(fe, value):
    dims = (20, 16, 24)
    face = fe_inputs.face_data(3, 9, *dims)
    sysm, x_or, x_star = reference(dims, face)
    s = fe.System(*dims, face_vals=torch.from_numpy(face).cuda()).build()
    x, res = solve_mixed(fe, s, "bcrs3", value)
    assert res.status == fe.FE_OK
    xg = x.cpu().numpy()
    assert oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg) <= 1.5e-10
    assert rel(xg, x_star) <= 2.0 * rel(x_or, x_star) + 1e-12


def test_mixed_edge_cases(fe):
    s = fe.System(6, 5, 4).build()
    # b = 0 gives x = 0 without an inner solve
    s.b.zero_()
    x, res = solve_mixed(fe, s, "bcrs3", "bf16")
    assert res.status == fe.FE_OK and res.outer_iterations == 0 and torch.count_nonzero(x) == 0
    s.build()
    # max_outer = 1 stops after one refinement step with MAXIT
    x, res = solve_mixed(fe, s, "csr", "bf16", max_outer=1)
    assert res.status == fe.FE_ERR_MAXIT and res.outer_iterations == 1
    assert 0 < res.relres < 1e-2
    # tol reachable only in FP64: FP32-valued matrix, tight tolerance, still converges
    x, res = solve_mixed(fe, s, "sell", "f32", tol=1e-13)
    assert res.status == fe.FE_OK and res.relres <= 1e-13
