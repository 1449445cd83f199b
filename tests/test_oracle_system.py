"""Pins for the oracle's mesh, matrix generation (Fig 3.6), assembly (Fig 3.7),
Dirichlet rows and SpMV (Fig 3.1, Fig 3.2), each against something other than
the oracle itself: closed forms, brute force, dense linear algebra.
"""
import itertools

import numpy as np
import pytest

import fe_inputs
import oracle


def node_xyz(nx, ny, nz):
    m = oracle.num_nodes(nx, ny, nz)
    i = np.arange(m)
    return i % (nx + 1), (i // (nx + 1)) % (ny + 1), i // ((nx + 1) * (ny + 1))


# --------------------------------------------------------------------------- mesh

def test_mesh_coords_and_default_bc():
    nx, ny, nz = 3, 4, 5
    coords, flag, val = oracle.mesh(nx, ny, nz)
    ix, iy, iz = node_xyz(nx, ny, nz)
    assert np.array_equal(coords[:, 0], ix / nx)
    assert np.array_equal(coords[:, 1], iy / ny)
    assert np.array_equal(coords[:, 2], iz / nz)
    on_b = (ix == 0) | (ix == nx) | (iy == 0) | (iy == ny) | (iz == 0) | (iz == nz)
    assert np.array_equal(flag.astype(bool), on_b)
    # paper Sec. 1: T = 1 on the plane x = 1, T = 0 on the other boundary planes
    assert np.array_equal(val, np.where(ix == nx, 1.0, 0.0))


def test_mesh_face_data_order():
    nx, ny, nz = 2, 3, 4
    fv = fe_inputs.face_data(7, 0, nx, ny, nz)
    assert fv.size == oracle.face_sizes(nx, ny, nz)
    coords, flag, val = oracle.mesh(nx, ny, nz, fv)
    ix, iy, iz = node_xyz(nx, ny, nz)
    nyz, nxz, nxy = (ny + 1) * (nz + 1), (nx + 1) * (nz + 1), (nx + 1) * (ny + 1)
    faces = np.split(fv, np.cumsum([nyz, nyz, nxz, nxz, nxy])[:])
    # z1 is applied last, so it owns its whole face
    sel = iz == nz
    assert np.array_equal(val[sel], faces[5][(ix + (nx + 1) * iy)[sel]])
    # an x0 node that lies on no other face keeps the x0 value
    sel = (ix == 0) & (iy > 0) & (iy < ny) & (iz > 0) & (iz < nz)
    assert np.array_equal(val[sel], faces[0][(iy + (ny + 1) * iz)[sel]])
    # y1 overwrites x1 on their shared edge (z interior)
    sel = (ix == nx) & (iy == ny) & (iz > 0) & (iz < nz)
    assert np.array_equal(val[sel], faces[3][(ix + (nx + 1) * iz)[sel]])
    assert np.all(val[flag == 0] == 0.0)


# --------------------------------------------------------------------------- pattern

@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 4), (4, 4, 4), (5, 2, 3), (30, 30, 30)])
def test_pattern_counts(dims):
    nx, ny, nz = dims
    row_ptr, cols = oracle.pattern(nx, ny, nz)
    nnz_closed = (3 * nx + 1) * (3 * ny + 1) * (3 * nz + 1)   # (3n-2) per axis, n = N+1 nodes
    assert row_ptr[-1] == cols.size == nnz_closed
    ix, iy, iz = node_xyz(nx, ny, nz)

    def axis_count(i, n):
        return np.where((i == 0) | (i == n), 2, 3) if n > 0 else np.ones_like(i)

    expect = axis_count(ix, nx) * axis_count(iy, ny) * axis_count(iz, nz)
    assert np.array_equal(np.diff(row_ptr), expect)
    if min(dims) >= 2:
        assert set(np.unique(np.diff(row_ptr))) == {8, 12, 18, 27}


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 2), (3, 3, 3)])
def test_pattern_brute_force(dims):
    nx, ny, nz = dims
    row_ptr, cols = oracle.pattern(nx, ny, nz)
    ix, iy, iz = node_xyz(nx, ny, nz)
    m = ix.size
    for i in range(m):
        nb = [j for j in range(m)
              if abs(ix[i] - ix[j]) <= 1 and abs(iy[i] - iy[j]) <= 1 and abs(iz[i] - iz[j]) <= 1]
        assert list(cols[row_ptr[i]:row_ptr[i + 1]]) == nb


def test_pattern_overflow_guard():
    with pytest.raises(OverflowError):
        oracle.pattern(430, 430, 430)   # (3*430+1)^3 > 2^31 - 1


# --------------------------------------------------------------------------- assembly

@pytest.mark.parametrize("n", [4, 8])
def test_assembled_interior_stencil(n):
    coords, flag, val = oracle.mesh(n, n, n)
    row_ptr, cols = oracle.pattern(n, n, n)
    vals, b = oracle.assemble(n, n, n, coords, row_ptr, cols)
    h = 1.0 / n
    assert np.all(b == 0.0)                       # no source term
    ix, iy, iz = node_xyz(n, n, n)
    # row sums vanish before boundary conditions (constants are harmonic)
    rs = np.add.reduceat(vals, row_ptr[:-1])
    assert np.abs(rs).max() < 1e-15
    expect = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}
    for i in np.nonzero(flag == 0)[0]:
        for k in range(row_ptr[i], row_ptr[i + 1]):
            j = cols[k]
            d = int(ix[i] != ix[j]) + int(iy[i] != iy[j]) + int(iz[i] != iz[j])
            assert abs(vals[k] - expect[d]) <= 1e-15 * h * 8, (i, j, d, vals[k])


def test_assembled_matrix_symmetric_and_brick_consistent():
    nx, ny, nz = 3, 2, 5
    sysm = oracle.build_system(nx, ny, nz)
    coords = sysm["coords"]
    row_ptr, cols = oracle.pattern(nx, ny, nz)
    vals, _ = oracle.assemble(nx, ny, nz, coords, row_ptr, cols)
    A = oracle.dense(row_ptr, cols, vals)
    assert np.allclose(A, A.T, atol=1e-15)
    # Kronecker structure of the trilinear Laplacian on a tensor grid:
    # A = Kx (x) My (x) Mz + ... with 1-D FE stiffness/mass matrices
    def k1(n):
        h = 1.0 / n
        K = np.zeros((n + 1, n + 1))
        for e in range(n):
            K[e:e + 2, e:e + 2] += np.array([[1, -1], [-1, 1]]) / h
        return K

    def m1(n):
        h = 1.0 / n
        M = np.zeros((n + 1, n + 1))
        for e in range(n):
            M[e:e + 2, e:e + 2] += np.array([[2, 1], [1, 2]]) * h / 6
        return M

    # node id = ix + (nx+1)(iy + (ny+1) iz): z is the slowest index
    ref = (np.kron(m1(nz), np.kron(m1(ny), k1(nx))) + np.kron(m1(nz), np.kron(k1(ny), m1(nx)))
           + np.kron(k1(nz), np.kron(m1(ny), m1(nx))))
    assert np.allclose(A, ref, atol=1e-14 * np.abs(ref).max())


# --------------------------------------------------------------------------- Dirichlet

@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 2), (8, 8, 8)])
def test_dirichlet_system_spd_and_equivalent(dims):
    nx, ny, nz = dims
    coords, flag, g = oracle.mesh(nx, ny, nz)
    row_ptr, cols = oracle.pattern(nx, ny, nz)
    K0, _ = oracle.assemble(nx, ny, nz, coords, row_ptr, cols)
    Kfull = oracle.dense(row_ptr, cols, K0)
    sysm = oracle.build_system(nx, ny, nz)
    A = oracle.dense(row_ptr, cols, sysm["vals"])
    b = sysm["b"]
    assert np.array_equal(row_ptr, sysm["row_ptr"]) and np.array_equal(cols, sysm["cols"])
    assert np.allclose(A, A.T, atol=0)
    np.linalg.cholesky(A)                       # SPD
    bnd = flag.astype(bool)
    assert np.array_equal(np.diag(A)[bnd], np.ones(bnd.sum()))
    assert np.array_equal(b[bnd], g[bnd])
    # the reduced system: K_II x_I = -K_IB g_B, x_B = g_B (textbook elimination)
    I, B = ~bnd, bnd
    xI = np.linalg.solve(Kfull[np.ix_(I, I)], -Kfull[np.ix_(I, B)] @ g[B])
    x = np.linalg.solve(A, b)
    assert np.allclose(x[I], xI, atol=1e-13)
    assert np.array_equal(x[B], g[B]) or np.allclose(x[B], g[B], atol=1e-15)


# --------------------------------------------------------------------------- SpMV

@pytest.mark.parametrize("dims", [(4, 4, 4), (2, 5, 3)])
def test_spmv_csr_matches_dense(dims):
    nx, ny, nz = dims
    sysm = oracle.build_system(nx, ny, nz)
    A = oracle.dense(sysm["row_ptr"], sysm["cols"], sysm["vals"])
    x = fe_inputs.random_vector(3, A.shape[0])
    y = oracle.spmv_csr(sysm["row_ptr"], sysm["cols"], sysm["vals"], x)
    assert np.allclose(y, A @ x, atol=1e-14)


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 2), (30, 30, 30)])
def test_bcrs_facts_and_spmv(dims):
    nx, ny, nz = dims
    sysm = oracle.build_system(nx, ny, nz)
    row_ptr, cols, vals = sysm["row_ptr"], sysm["cols"], sysm["vals"]
    ptr, jas, offsets = oracle.csr_to_bcrs(row_ptr, cols)
    nns = jas.size
    lens = np.diff(offsets)
    # single domain with >= 4 nodes per x-line: every x-run has 2 or 3 nodes
    assert set(np.unique(lens)) <= {2, 3}
    assert nns == (nx + 1) * (3 * ny + 1) * (3 * nz + 1)
    # segments of length 3 are the share (n-2)/n of each x-line, n = nx+1 nodes
    assert np.isclose(np.mean(lens == 3), (nx - 1) / (nx + 1))
    # paper Sec. 3.1: nnz = sum of segment lengths; memory access counts
    assert lens.sum() == cols.size
    nnz, m = cols.size, row_ptr.size - 1
    crs_access, bcrs_access = 3 * nnz + 2 * m + 1, 2 * nnz + 2 * nns + 2 * m + 2
    assert crs_access - bcrs_access == nnz - 2 * nns - 1
    # Fig 3.2 SpMV: same per-row summation order as Fig 3.1, so identical bits
    x = fe_inputs.random_vector(5, m)
    assert np.array_equal(oracle.spmv_bcrs(ptr, jas, offsets, vals, x),
                          oracle.spmv_csr(row_ptr, cols, vals, x))


def test_bcrs_runs_merge_across_short_lines():
    """With 3 nodes per x-line a middle row covers the whole line, and the next
    line's first node is both adjacent in id and a stencil neighbour, so the
    maximal runs of Sec. 3.1 span two lines (lengths 6 and 9 appear)."""
    sysm = oracle.build_system(2, 3, 3)
    ptr, jas, offsets = oracle.csr_to_bcrs(sysm["row_ptr"], sysm["cols"])
    lens = np.diff(offsets)
    assert lens.max() > 3 and lens.sum() == sysm["cols"].size
    x = fe_inputs.random_vector(9, sysm["b"].size)
    assert np.array_equal(oracle.spmv_bcrs(ptr, jas, offsets, sysm["vals"], x),
                          oracle.spmv_csr(sysm["row_ptr"], sysm["cols"], sysm["vals"], x))
