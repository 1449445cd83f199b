"""Pins of the oracle's closed-form extreme eigenvalues of the Dirichlet system
(identity rows on boundary nodes, Kronecker-sum interior block of the brick
element) -- the lambda_min behind the forward-error bars of the solver tests:
||x - x*|| <= ||b - A x|| / lambda_min(A) for any x.

Checked against the dense symmetric eigensolver on the oracle's assembled
matrix (element integrals, scatter, Dirichlet elimination), so a wrong 1D
eigenvalue, a dropped Kronecker term or a missing identity row fails.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 3, 4), (2, 2, 2), (6, 2, 3), (1, 3, 3),
                                  (3, 7, 2), (7, 7, 6)])
def test_extreme_eigenvalues_match_dense_solver(dims):
    s = oracle.build_system(*dims)
    A = oracle.dense(s["row_ptr"], s["cols"], s["vals"])
    assert np.abs(A - A.T).max() <= 1e-15
    ev = np.linalg.eigvalsh(A)
    lo, hi = oracle.dirichlet_extreme_eigenvalues(*dims)
    assert abs(ev.min() - lo) <= 1e-13 * lo
    assert abs(ev.max() - hi) <= 1e-13 * hi


def test_smallest_eigenvalue_continuum_limit():
    """h^-3 lambda_min -> 3 pi^2 (the Laplacian's first Dirichlet eigenvalue on the
    unit cube, times the mass scaling h^3), at O(h^2)."""
    errs = []
    for n in (16, 32, 64):
        lo, hi = oracle.dirichlet_extreme_eigenvalues(n, n, n)
        assert hi == 1.0                  # the boundary rows' identity dominates
        errs.append(abs(lo * n ** 3 - 3 * np.pi ** 2))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_forward_error_bound_holds_for_oracle_iterates():
    """The bound the mixed-precision and batched tests use, on the oracle's own CG
    iterates: ||x_k - x*|| <= ||b - A x_k|| / lambda_min at every checked step."""
    dims = (9, 8, 7)
    s = oracle.build_system(*dims)
    lo, _ = oracle.dirichlet_extreme_eigenvalues(*dims)
    A = oracle.dense(s["row_ptr"], s["cols"], s["vals"])
    xs = np.linalg.solve(A, s["b"])
    for k in (1, 5, 20, 40):
        xk, _, _, _ = oracle.cg(s["row_ptr"], s["cols"], s["vals"], s["b"], tol=0.0, maxit=k)
        r = s["b"] - A @ xk
        assert np.linalg.norm(xk - xs) <= np.linalg.norm(r) / lo * (1 + 1e-12)
