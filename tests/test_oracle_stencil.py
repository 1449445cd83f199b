"""Pins of the oracle's matrix-free operator (the same Dirichlet system as the
assembled one, applied from the brick element's Kronecker structure).

Each pin checks it against something other than itself: the closed-form cube
stencil (8h/3, 0, -h/6, -h/12), the element-integral assembly of the oracle
(Gauss quadrature, Fig 3.7 scatter, Dirichlet elimination), and a dense
Kronecker sum built here with numpy from 1D linear elements.
"""
import numpy as np
import pytest

import fe_inputs
import oracle

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n", [2, 3, 8, 30, 256])
def test_cube_stencil_closed_form(n):
    h = 1.0 / n
    a = oracle.stencil_coeffs(n, n, n)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                d = (dx != 1) + (dy != 1) + (dz != 1)
                want = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[d]
                assert abs(a[dz, dy, dx] - want) <= 8 * EPS * h, (dx, dy, dz)


@pytest.mark.parametrize("dims", [(4, 3, 5), (2, 7, 3), (9, 9, 2)])
def test_brick_stencil_row_sums_symmetry_signs(dims):
    a = oracle.stencil_coeffs(*dims)
    h = 1.0 / min(dims)
    assert abs(a.sum()) <= 64 * EPS / h        # constants are in the kernel
    assert np.array_equal(a, a[::-1, ::-1, ::-1])   # a(d) = a(-d)
    assert a[1, 1, 1] > 0
    # on a stretched brick face and edge entries can be positive (the
    # trilinear stencil is not an M-matrix there); each corner entry is a sum
    # of three products M(1) M(1) L(1) < 0
    for dz in (0, 2):
        for dy in (0, 2):
            for dx in (0, 2):
                assert a[dz, dy, dx] < 0


def _row_scale(sysm):
    rp, vals = sysm["row_ptr"], np.abs(sysm["vals"])
    return np.array([vals[rp[i]:rp[i + 1]].max() for i in range(rp.size - 1)])


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (4, 4, 4), (3, 5, 2), (6, 2, 7), (9, 8, 10)])
def test_stencil_matches_assembled_operator(dims):
    sysm = oracle.build_system(*dims)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(sysm["b"].size)
    y_csr = oracle.spmv_csr(sysm["row_ptr"], sysm["cols"], sysm["vals"], x)
    y_mf = oracle.stencil_spmv(*dims, x)
    scale = _row_scale(sysm) * np.abs(x).max()
    assert (np.abs(y_csr - y_mf) <= 1e-13 * scale).all()
    for i in rng.integers(0, x.size, 20):
        assert oracle.stencil_row(*dims, int(i), x) == y_mf[i]


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 3, 6), (8, 8, 8)])
@pytest.mark.parametrize("faces", ["paper", "random"])
def test_stencil_rhs_matches_assembled(dims, faces):
    face = None if faces == "paper" else fe_inputs.face_data(0, 3, *dims)
    sysm = oracle.build_system(*dims, face)
    b = oracle.stencil_rhs(*dims, sysm["bc_val"])
    scale = _row_scale(sysm) * max(1.0, np.abs(sysm["bc_val"]).max())
    assert (np.abs(b - sysm["b"]) <= 1e-13 * scale).all()
    assert np.array_equal(b[sysm["bc_flag"] == 1], sysm["bc_val"][sysm["bc_flag"] == 1])


def _assembled_1d(n):
    """Assembled 1D linear-element mass and stiffness on n elements of [0, 1]."""
    h = 1.0 / n
    M = np.zeros((n + 1, n + 1))
    L = np.zeros((n + 1, n + 1))
    me = h * np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    le = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    for e in range(n):
        M[e:e + 2, e:e + 2] += me
        L[e:e + 2, e:e + 2] += le
    return M, L


@pytest.mark.parametrize("dims", [(3, 4, 2), (5, 5, 5), (1, 3, 4)])
def test_stencil_equals_dense_kronecker_sum(dims):
    nx, ny, nz = dims
    Mx, Lx = _assembled_1d(nx)
    My, Ly = _assembled_1d(ny)
    Mz, Lz = _assembled_1d(nz)
    # node id = ix + (nx+1)(iy + (ny+1) iz): x is the fastest, so the last factor
    A = (np.kron(Mz, np.kron(My, Lx)) + np.kron(Mz, np.kron(Ly, Mx)) +
         np.kron(Lz, np.kron(My, Mx)))
    _, flag, _ = oracle.mesh(*dims)
    bc = flag.astype(bool)
    A[bc, :] = 0.0
    A[:, bc] = 0.0
    A[bc, bc] = 1.0
    x = np.random.default_rng(5).standard_normal(A.shape[0])
    assert np.allclose(oracle.stencil_spmv(*dims, x), A @ x, rtol=0, atol=1e-13)
