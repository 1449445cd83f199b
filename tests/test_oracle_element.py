"""Pins for the oracle's element operator (paper Sec. 1, "element operator
computing"): the 8x8 hexahedral diffusion matrix from 2x2x2 Gauss quadrature.

Independent of the oracle's code path:
  * cube of side h: exact closed form (h/12) * [4, 0, -1, -1] indexed by the
    number of corner coordinates in which nodes a and b differ;
  * brick hx x hy x hz: Kronecker sum of exact 1-D stiffness and mass matrices;
  * sheared parallelepiped: exact reference-cell integrals of shape-function
    derivative products contracted with (J^T J)^{-1} det J (catches a
    transposed Jacobian);
  * symmetry and zero row sums (constants lie in the kernel of the Laplacian).
"""
import itertools

import numpy as np
import pytest

import oracle

CORNERS = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                    (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)])


def cube_closed_form(h):
    c = {0: 4.0, 1: 0.0, 2: -1.0, 3: -1.0}
    K = np.empty((8, 8))
    for a in range(8):
        for b in range(8):
            d = int(np.sum(CORNERS[a] != CORNERS[b]))
            K[a, b] = h / 12.0 * c[d]
    return K


def brick_closed_form(hx, hy, hz):
    def k1(h):
        return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h

    def m1(h):
        return np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0

    K = np.empty((8, 8))
    for a in range(8):
        for b in range(8):
            ia, ib = CORNERS[a], CORNERS[b]
            K[a, b] = (k1(hx)[ia[0], ib[0]] * m1(hy)[ia[1], ib[1]] * m1(hz)[ia[2], ib[2]]
                       + m1(hx)[ia[0], ib[0]] * k1(hy)[ia[1], ib[1]] * m1(hz)[ia[2], ib[2]]
                       + m1(hx)[ia[0], ib[0]] * m1(hy)[ia[1], ib[1]] * k1(hz)[ia[2], ib[2]])
    return K


def parallelepiped_closed_form(origin, J):
    """K for x = origin + J (xi+1)/2 ... with J the constant Jacobian d x / d xi."""
    # 1-D linear shape functions on [-1, 1]: phi_0 = (1-xi)/2, phi_1 = (1+xi)/2
    mass = np.array([[2 / 3, 1 / 3], [1 / 3, 2 / 3]])       # int phi_a phi_b
    stiff = np.array([[0.5, -0.5], [-0.5, 0.5]])           # int phi_a' phi_b'
    dphi = np.array([-0.5, 0.5])
    mixed = np.array([[dphi[a] * 1.0 for b in range(2)] for a in range(2)])  # int phi_a' phi_b

    def one_d(a, b, da, db):
        if da and db:
            return stiff[a, b]
        if da:
            return mixed[a, b]
        if db:
            return mixed[b, a]
        return mass[a, b]

    G = np.linalg.inv(J.T @ J)
    det = np.linalg.det(J)
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            for i in range(3):
                for j in range(3):
                    integral = 1.0
                    for ax in range(3):
                        integral *= one_d(CORNERS[a][ax], CORNERS[b][ax], ax == i, ax == j)
                    K[a, b] += G[i, j] * integral
            K[a, b] *= det
    return K


@pytest.mark.parametrize("h", [1.0, 0.25, 1.0 / 30, 1.0 / 256])
def test_cube_matches_closed_form(h):
    X = CORNERS * h + np.array([0.3, -1.0, 2.0]) * h
    K = oracle.element_matrix(X)
    ref = cube_closed_form(h)
    assert np.allclose(K, ref, rtol=0, atol=4e-15 * h)


@pytest.mark.parametrize("hx,hy,hz", [(0.5, 0.25, 0.125), (1.0 / 30, 1.0 / 7, 1.0 / 3)])
def test_brick_matches_kronecker_form(hx, hy, hz):
    X = CORNERS * np.array([hx, hy, hz])
    K = oracle.element_matrix(X)
    ref = brick_closed_form(hx, hy, hz)
    assert np.allclose(K, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


def test_sheared_parallelepiped():
    J = np.array([[0.6, 0.2, 0.05], [0.0, 0.5, 0.15], [0.1, 0.0, 0.7]]) * 0.5
    origin = np.array([0.1, 0.2, 0.3])
    xi = 2.0 * CORNERS - 1.0
    X = origin + (xi + 1.0) @ J.T
    K = oracle.element_matrix(X)
    ref = parallelepiped_closed_form(origin, J)
    assert np.allclose(K, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    # the transposed metric gives a different matrix here, so the pin is sharp
    Gt = parallelepiped_closed_form(origin, J.T)
    assert np.abs(Gt - ref).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_symmetric_zero_rowsum_psd(seed):
    g = np.random.default_rng(seed)
    X = CORNERS * 0.1 + g.uniform(-0.015, 0.015, size=(8, 3))
    K = oracle.element_matrix(X)
    scale = np.abs(K).max()
    assert np.allclose(K, K.T, atol=1e-15 * scale)
    assert np.abs(K.sum(axis=1)).max() < 1e-14 * scale
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert ev.min() > -1e-13 * scale           # one zero mode (constants), rest > 0
    assert np.sum(ev > 1e-8 * scale) == 7


def test_element_nodes_local_order():
    nx, ny, nz = 3, 2, 4
    e = 1 + nx * (1 + ny * 2)          # element (1, 1, 2)
    nodes = oracle.element_nodes(nx, ny, nz, e)
    for a, (ox, oy, oz) in enumerate(CORNERS):
        ix, iy, iz = 1 + ox, 1 + oy, 2 + oz
        assert nodes[a] == ix + (nx + 1) * (iy + (ny + 1) * iz)
