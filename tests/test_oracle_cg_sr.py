"""Pins for the oracle's single-reduction CG (Chronopoulos-Gear recurrences):
Krylov termination on matrices with few distinct eigenvalues (a dropped or
mis-signed term in beta, the curvature recurrence or the s recurrence breaks
it), agreement with textbook CG step by step, a dense direct solve, and the
status codes."""
import numpy as np
import pytest

import fe_inputs
import oracle


def diag_csr(d):
    m = len(d)
    return (np.arange(m + 1, dtype=np.int32), np.arange(m, dtype=np.int32),
            np.asarray(d, dtype=np.float64))


def sym_csr(A):
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(A.shape[0] + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), cols.astype(np.int32), A[rows, cols].astype(np.float64)


@pytest.mark.parametrize("eigs", [(1.0, 3.0), (0.5, 2.0, 7.0), (1.0, 2.0, 4.0, 9.0)])
def test_krylov_termination(eigs):
    """Exact arithmetic: k distinct eigenvalues -> solved after k steps.  A
    rotated diagonal (dense SPD matrix) so every entry of the recurrences is
    exercised; rounding leaves a residual near machine precision."""
    g = np.random.default_rng(1)
    m = 12
    d = np.array([eigs[i % len(eigs)] for i in range(m)])
    Q, _ = np.linalg.qr(g.standard_normal((m, m)))
    A = Q @ np.diag(d) @ Q.T
    A = 0.5 * (A + A.T)
    rp, cols, vals = sym_csr(A)
    b = g.standard_normal(m)
    x, it, rel, st = oracle.cg_sr(rp, cols, vals, b, tol=1e-12, maxit=50)
    assert st == oracle.CG_CONVERGED
    assert it == len(eigs)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    # one step before termination the residual is far from zero
    _, it2, rel2, st2 = oracle.cg_sr(rp, cols, vals, b, tol=1e-12, maxit=len(eigs) - 1)
    assert st2 == oracle.CG_MAXIT and rel2 > 1e-6


def test_iterates_match_textbook_cg():
    face = fe_inputs.face_data(21, 0, 6, 5, 7)
    s = oracle.build_system(6, 5, 7, face)
    rp, cols, vals, b = s["row_ptr"], s["cols"], s["vals"], s["b"]
    for k in range(1, 9):
        x1, i1, r1, _ = oracle.cg(rp, cols, vals, b, tol=0.0, maxit=k)
        x2, i2, r2, _ = oracle.cg_sr(rp, cols, vals, b, tol=0.0, maxit=k)
        assert i1 == i2 == k
        assert np.linalg.norm(x2 - x1) <= 1e-12 * np.linalg.norm(x1)
        assert abs(r2 - r1) <= 1e-10 * r1


def test_dense_direct_solve_and_stop_count():
    face = fe_inputs.face_data(22, 0, 8, 8, 8)
    s = oracle.build_system(8, 8, 8, face)
    rp, cols, vals, b = s["row_ptr"], s["cols"], s["vals"], s["b"]
    A = oracle.dense(rp, cols, vals)
    xd = np.linalg.solve(A, b)
    x, it, rel, st = oracle.cg_sr(rp, cols, vals, b, tol=1e-12, maxit=1000)
    _, it_tb, _, _ = oracle.cg(rp, cols, vals, b, tol=1e-12, maxit=1000)
    assert st == oracle.CG_CONVERGED and abs(it - it_tb) <= 1
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert oracle.true_relres(rp, cols, vals, b, x) <= 2e-12


def test_status_codes():
    rp, cols, vals = diag_csr([1.0, 2.0, 3.0])
    x, it, rel, st = oracle.cg_sr(rp, cols, vals, np.zeros(3), x0=np.ones(3))
    assert st == oracle.CG_CONVERGED and it == 0 and not x.any()
    _, it, _, st = oracle.cg_sr(rp, cols, vals, np.ones(3), tol=0.0, maxit=1)
    assert st == oracle.CG_MAXIT and it == 1
    rp, cols, vals = diag_csr([1.0, -1.0])
    _, _, _, st = oracle.cg_sr(rp, cols, vals, np.array([1.0, 1.0]))
    assert st == oracle.CG_BREAKDOWN
    # converged start vector: no step taken
    rp, cols, vals = diag_csr([2.0, 4.0])
    _, it, _, st = oracle.cg_sr(rp, cols, vals, np.array([2.0, 4.0]), x0=np.ones(2))
    assert st == oracle.CG_CONVERGED and it == 0


def test_restart_when_the_curvature_recurrence_is_not_positive():
    """diag(3, -1), b = (1, 1), worked by hand.  Step 1: r0 = b, delta = 2,
    alpha = 1, x1 = (1, 1), r1 = (-2, 2), gamma = 8, w1 = A r1 = (-6, -2),
    delta = 8.  Step 2: beta = 4 and the recurrence gives p.Ap = 8 - 4*8/1 = -24
    (textbook CG breaks down here: p = (2, 6), p.Ap = -24); the single-reduction
    form restarts the direction: p = r1, alpha = gamma / delta = 1,
    x2 = x1 + r1 = (-1, 3)."""
    rp, cols, vals = diag_csr([3.0, -1.0])
    b = np.array([1.0, 1.0])
    _, _, _, st = oracle.cg(rp, cols, vals, b, tol=1e-12, maxit=2)
    assert st == oracle.CG_BREAKDOWN
    x, it, rel, st = oracle.cg_sr(rp, cols, vals, b, tol=1e-12, maxit=2)
    assert st == oracle.CG_MAXIT and it == 2
    assert np.array_equal(x, np.array([-1.0, 3.0]))
    _, it, _, _ = oracle.cg_sr(rp, cols, vals, b, tol=1e-12, maxit=1)
    x1, _, _, _ = oracle.cg_sr(rp, cols, vals, b, tol=0.0, maxit=1)
    assert np.array_equal(x1, np.array([1.0, 1.0]))
