"""GPU parity of the single-reduction CG (fe_cg_solve_sr, Chronopoulos-Gear
recurrences) against the oracle's single-reduction CG, through the C ABI.

Same criteria as the textbook solver (test_gpu_cg.py): the GPU reduces dot
products in a blocked order, CG amplifies that rounding, so
  (i)   stop iteration within +-1 of the oracle's;
  (ii)  ||x_gpu - x*|| <= 2 ||x_oracle - x*|| + 1e-12 ||x*|| at tol 1e-10,
        x* the oracle's textbook solve to 1e-14;
  (iii) the oracle's true relative residual of x_gpu <= 1.5e-10;
  (iv)  solved to 1e-12 on both sides, ||x_gpu - x_oracle|| <= 1e-10 ||x_oracle||.
"""
import time

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


def solve_sr(fe, s, fmt, tol=1e-10, maxit=1000, x0=None, b=None, timeout=0.0, check=True):
    A = s.matrix(fmt, "f64")
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda") if x0 is None else x0.clone()
    work = fe.sr_workspace(A)
    res = fe.fe_cg_solve_sr(A.desc, s.b if b is None else b, x, tol, maxit, work, timeout,
                            check=check)
    return x, res


REF = {}


def reference(dims, face=None, tol=1e-10):
    key = (dims, None if face is None else face.tobytes(), tol)
    if key not in REF:
        sysm = oracle.build_system(*dims, face)
        x, it, rel, st = oracle.cg_sr(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                      tol=tol, maxit=5000)
        xs, _, _, _ = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                tol=1e-14, maxit=20000)
        REF[key] = (sysm, it, st, x, xs)
    return REF[key]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_parity(ref, x_gpu, k_gpu, tol=1e-10):
    sysm, k_ref, st, x_or, x_star = ref
    assert abs(k_gpu - k_ref) <= 1, (k_gpu, k_ref)
    assert rel(x_gpu, x_star) <= 2.0 * rel(x_or, x_star) + 1e-12
    tr = oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], x_gpu)
    assert tr <= 1.5 * tol


@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("dims", [(30, 30, 30), (4, 4, 4), (17, 9, 23)])
def test_sr_parity(fe, fmt, dims):
    ref = reference(dims)
    assert ref[2] == oracle.CG_CONVERGED
    s = fe.System(*dims).build()
    x, res = solve_sr(fe, s, fmt)
    assert res.status == fe.FE_OK and res.relres <= 1e-10
    check_parity(ref, x.cpu().numpy(), res.iterations)


@pytest.mark.parametrize("fmt", ["csr", "bcrs3"])
def test_sr_solution_parity_tight(fe, fmt):
    dims = (30, 30, 30)
    ref = reference(dims, tol=1e-12)
    s = fe.System(*dims).build()
    x, res = solve_sr(fe, s, fmt, tol=1e-12)
    assert res.status == fe.FE_OK and abs(res.iterations - ref[1]) <= 1
    assert rel(x.cpu().numpy(), ref[3]) <= 1e-10


def test_sr_face_data_and_nonzero_start(fe):
    dims = (24, 20, 16)
    face = fe_inputs.face_data(3, 1, *dims)
    ref = reference(dims, face)
    s = fe.System(*dims, face_vals=torch.from_numpy(face).cuda()).build()
    x, res = solve_sr(fe, s, "sell")
    assert res.status == fe.FE_OK
    check_parity(ref, x.cpu().numpy(), res.iterations)
    # from a non-zero start: the oracle from the same start
    g = np.random.default_rng(4)
    x0 = g.standard_normal(s.m)
    sysm = ref[0]
    xo, ito, _, sto = oracle.cg_sr(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], x0=x0,
                                   tol=1e-12, maxit=5000)
    x, res = solve_sr(fe, s, "bcrs3", tol=1e-12, x0=torch.from_numpy(x0).cuda())
    assert res.status == fe.FE_OK and abs(res.iterations - ito) <= 1
    assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_sr_matches_textbook_gpu_solver(fe):
    """Same Krylov method: step counts within 1, solutions as accurate."""
    s = fe.System(30).build()
    A = s.matrix("bcrs3")
    x1 = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    r1 = fe.fe_cg_solve(A.desc, s.b, x1, 1e-10, 1000, fe.cg_workspace(A))
    x2, r2 = solve_sr(fe, s, "bcrs3")
    assert abs(r1.iterations - r2.iterations) <= 1
    work = fe.resid_workspace()
    assert fe.fe_true_relres(A.desc, s.b, x2, work) <= 1.5e-10


def test_sr_bitwise_repeatable(fe):
    s = fe.System(30).build()
    x1, r1 = solve_sr(fe, s, "bcrs3")
    x2, r2 = solve_sr(fe, s, "bcrs3")
    assert r1.iterations == r2.iterations and r1.relres == r2.relres
    assert torch.equal(x1, x2)


def test_sr_edge_cases(fe):
    s = fe.System(6, 5, 4).build()
    zero = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    x, res = solve_sr(fe, s, "bcrs3", b=zero, x0=torch.ones_like(zero))
    assert res.status == fe.FE_OK and res.iterations == 0 and torch.count_nonzero(x) == 0
    x, res = solve_sr(fe, s, "csr", maxit=3, check=False)
    assert res.status == fe.FE_ERR_MAXIT and res.iterations == 3
    sysm = oracle.build_system(6, 5, 4)
    x3, _, _, _ = oracle.cg_sr(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], tol=0, maxit=3)
    assert np.allclose(x.cpu().numpy(), x3, rtol=0, atol=1e-12)
    x, res = solve_sr(fe, s, "sell", maxit=0, check=False)
    assert res.status == fe.FE_ERR_MAXIT and res.iterations == 0
    xs, res = solve_sr(fe, s, "bcrs3", tol=1e-13)
    x, res = solve_sr(fe, s, "bcrs3", x0=xs, tol=1e-10)
    assert res.status == fe.FE_OK and res.iterations == 0
    bn = s.b.clone()
    bn[s.m // 2] = float("nan")
    x, res = solve_sr(fe, s, "csr", b=bn, check=False)
    assert res.status == fe.FE_ERR_BREAKDOWN
    t = fe.System(1).build()
    x, res = solve_sr(fe, t, "bcrs3")
    assert res.status == fe.FE_OK and res.iterations <= 1
    assert torch.equal(x, t.bc_val)


def test_sr_indefinite_breaks_down(fe):
    s = fe.System(5).build()
    sysm = oracle.build_system(5, 5, 5)
    rp, c = sysm["row_ptr"], sysm["cols"]
    diag = np.array([k for i in range(rp.size - 1) for k in range(rp[i], rp[i + 1]) if c[k] == i])
    s.vals[torch.from_numpy(diag).cuda()] *= -1.0
    s.drop_formats()
    x, res = solve_sr(fe, s, "csr", check=False)
    assert res.status == fe.FE_ERR_BREAKDOWN


def test_sr_barrier_timeout_is_reported_and_context_survives(fe):
    s = fe.System(16).build()
    fe.fe_inject_barrier_stall(5)
    t0 = time.time()
    x, res = solve_sr(fe, s, "bcrs3", timeout=0.2, check=False)
    assert res.status == fe.FE_ERR_TIMEOUT and time.time() - t0 < 10.0
    x, res = solve_sr(fe, s, "bcrs3")
    assert res.status == fe.FE_OK


@pytest.mark.slow
def test_sr_full_size_n256(fe):
    s = fe.System(256).build()
    x, res = solve_sr(fe, s, "bcrs3", maxit=2000)
    assert res.status == fe.FE_OK and 450 <= res.iterations <= 650
    tr = fe.fe_true_relres(s.matrix("csr").desc, s.b, x, fe.resid_workspace())
    assert tr <= 1.5e-10
    centre = 128 + 257 * (128 + 257 * 128)
    assert abs(float(x[centre]) - 1.0 / 6.0) < 2e-5
