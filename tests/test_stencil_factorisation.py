"""The plane-sum factorisation the matrix-free kernel evaluates, checked on
the CPU against the oracle's 27-point operator: for interior rows

    y = c0 X + c1 Sx + c2 Sy + c3 D   (plane z)  +  Q(z-1) + Q(z+1),
    Q = c4 X + c5 Sx + c6 Sy + c7 D,

with X the centre, Sx / Sy the in-plane axis neighbour sums, D the in-plane
diagonal sum (= Sx of the rows above and below) and c[k] the coefficient of
class k = |dx| + 2|dy| + 4|dz|; on a cube c1 = c2 = c4 = 0 and the edge
classes agree, so y = c0 X + c3 D + P(z-1) + P(z+1), P = c3 (Sx + Sy) + c7 D.
Boundary columns read as 0, boundary rows are identity rows."""
import numpy as np
import pytest

import oracle


def factorised(dims, x, cube):
    nx, ny, nz = dims
    a = oracle.stencil_coeffs(*dims)
    c = np.array([a[1 + (k >> 2), 1 + ((k >> 1) & 1), 1 + (k & 1)] for k in range(8)])
    X = x.reshape(nz + 1, ny + 1, nx + 1).copy()
    _, flag, _ = oracle.mesh(*dims)
    bnd = flag.reshape(X.shape).astype(bool)
    Xt = np.where(bnd, 0.0, X)                     # eliminated boundary columns
    P = np.pad(Xt, 1)
    Sx = P[1:-1, 1:-1, :-2] + P[1:-1, 1:-1, 2:]
    Sy = P[1:-1, :-2, 1:-1] + P[1:-1, 2:, 1:-1]
    SxP = np.pad(Sx, ((0, 0), (1, 1), (0, 0)))
    D = SxP[:, :-2, :] + SxP[:, 2:, :]               # Sx of the rows above and below
    if cube:
        Q = c[3] * (Sx + Sy) + c[7] * D
        inplane = c[0] * Xt + c[3] * D
    else:
        Q = c[4] * Xt + c[5] * Sx + c[6] * Sy + c[7] * D
        inplane = c[0] * Xt + c[1] * Sx + c[2] * Sy + c[3] * D
    QP = np.pad(Q, ((1, 1), (0, 0), (0, 0)))
    y = inplane + QP[:-2] + QP[2:]
    y = np.where(bnd, X, y)                          # identity rows
    return y.ravel()


@pytest.mark.parametrize("dims,cube", [((6, 6, 6), True), ((17, 17, 17), True), ((5, 7, 4), False),
                                       ((9, 3, 12), False), ((1, 1, 1), True), ((2, 5, 3), False)])
def test_plane_sum_factorisation_equals_the_operator(dims, cube):
    m = oracle.num_nodes(*dims)
    x = np.random.default_rng(3).standard_normal(m)
    want = oracle.stencil_spmv(*dims, x)
    got = factorised(dims, x, cube)
    scale = np.abs(oracle.stencil_coeffs(*dims)).sum() * np.abs(x).max()
    assert np.abs(got - want).max() <= 1e-14 * scale
