"""GPU parity of mesh processing, matrix generation and assembly against the
CPU oracle, through the C ABI.

Bars: coordinates, boundary data, row pointer and columns bit-exact; matrix
values and right-hand side within 1e-14 of the row's largest |a_ij|, on box
meshes (parallelepipeds: the constant-Jacobian path), sheared meshes of
exact binary coordinates (the same path with a full Jacobian) and meshes with
moved interior nodes (the per-point quadrature path) (each
entry sums <= 8 element contributions, each a Gauss sum of O(100) roundings,
so about 45 ulp of the row scale; entries that are zero in exact arithmetic
come out near 1e-18 and are covered by the row scale).
"""
import numpy as np
import pytest
import torch

import fe_inputs
import oracle

pytestmark = pytest.mark.gpu

VAL_TOL = 1e-14


@pytest.fixture(scope="module")
def fe():
    import paper_1505_08023_gb300.fe as fe_mod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    fe_mod.load()
    return fe_mod


def gpu_system(fe, dims, face=None):
    fv = None if face is None else torch.from_numpy(face).cuda()
    s = fe.System(*dims, face_vals=fv, keep_conn=True).build()
    torch.cuda.synchronize()
    return s


def host(t):
    return t.cpu().numpy()


def row_scaled_close(row_ptr, ref, got, tol=VAL_TOL):
    scale = np.maximum.reduceat(np.abs(ref), row_ptr[:-1])
    rows = np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr))
    err = np.abs(got - ref) / scale[rows]
    return err.max()


DIMS = [(1, 1, 1), (2, 3, 4), (4, 4, 4), (7, 3, 5), (30, 30, 30), (33, 17, 9)]


@pytest.mark.parametrize("dims", DIMS)
def test_mesh_and_pattern_bit_exact(fe, dims):
    s = gpu_system(fe, dims)
    coords, flag, val = oracle.mesh(*dims)
    assert np.array_equal(host(s.coords), coords)
    assert np.array_equal(host(s.bc_flag), flag)
    assert np.array_equal(host(s.bc_val), val)
    row_ptr, cols = oracle.pattern(*dims)
    assert np.array_equal(host(s.row_ptr), row_ptr)
    assert np.array_equal(host(s.cols), cols)
    conn = host(s.conn)
    for e in [0, conn.shape[0] // 2, conn.shape[0] - 1]:
        assert np.array_equal(conn[e], oracle.element_nodes(*dims, e))


@pytest.mark.parametrize("dims", DIMS)
def test_assembled_values_and_rhs(fe, dims):
    s = gpu_system(fe, dims)
    ref = oracle.build_system(*dims)
    vals = host(s.vals)
    assert row_scaled_close(ref["row_ptr"], ref["vals"], vals) <= VAL_TOL
    bscale = max(np.abs(ref["b"]).max(), 1.0)
    assert np.abs(host(s.b) - ref["b"]).max() <= VAL_TOL * bscale
    # Dirichlet rows are exact identity rows on both sides
    bnd = ref["bc_flag"].astype(bool)
    rp = ref["row_ptr"]
    for i in np.nonzero(bnd)[0][:50]:
        assert np.array_equal(vals[rp[i]:rp[i + 1]], ref["vals"][rp[i]:rp[i + 1]])


@pytest.mark.parametrize("dims", [(4, 4, 4), (9, 6, 5), (30, 30, 30)])
def test_face_data_assembly(fe, dims):
    face = fe_inputs.face_data(123, 4, *dims)
    s = gpu_system(fe, dims, face)
    coords, flag, val = oracle.mesh(*dims, face)
    assert np.array_equal(host(s.bc_val), val)
    ref = oracle.build_system(*dims, face)
    assert row_scaled_close(ref["row_ptr"], ref["vals"], host(s.vals)) <= VAL_TOL
    assert np.abs(host(s.b) - ref["b"]).max() <= VAL_TOL * max(np.abs(ref["b"]).max(), 1.0)


def _assemble_with_coords(fe, dims, X):
    """GPU assembly from the given node coordinates, and the oracle's."""
    s = fe.System(*dims)
    s.generate_mesh()
    s.coords.copy_(torch.from_numpy(X))
    s.assemble()
    _, flag, val = oracle.mesh(*dims)
    row_ptr, cols = oracle.pattern(*dims)
    vals, b = oracle.assemble(*dims, X, row_ptr, cols)
    oracle.dirichlet(flag, val, row_ptr, cols, vals, b)
    return s, row_ptr, vals, b


@pytest.mark.parametrize("dims", [(5, 4, 3), (12, 9, 7)])
def test_assembly_of_distorted_elements(fe, dims):
    """Interior nodes moved at random: trilinear elements with a varying
    Jacobian (the per-point quadrature path of the element kernel)."""
    coords, flag, _ = oracle.mesh(*dims)
    rng = np.random.default_rng(7)
    X = coords.copy()
    inner = ~flag.astype(bool)
    X[inner] += (0.2 / max(dims)) * rng.uniform(-1.0, 1.0, (int(inner.sum()), 3))
    s, row_ptr, vals, b = _assemble_with_coords(fe, dims, X)
    assert row_scaled_close(row_ptr, vals, host(s.vals)) <= VAL_TOL
    assert np.abs(host(s.b) - b).max() <= VAL_TOL * max(np.abs(b).max(), 1.0)


def test_assembly_of_sheared_parallelepipeds(fe):
    """A sheared mesh whose coordinates are exact binary fractions, so every
    element is a parallelepiped bit for bit (the constant-Jacobian path with
    a full, non-diagonal Jacobian)."""
    dims = (8, 8, 8)
    coords, _, _ = oracle.mesh(*dims)
    X = coords.copy()
    X[:, 0] = coords[:, 0] + 0.5 * coords[:, 1] + 0.25 * coords[:, 2]
    X[:, 1] = coords[:, 1] + 0.5 * coords[:, 2]
    X[:, 2] = 0.75 * coords[:, 2]
    s, row_ptr, vals, b = _assemble_with_coords(fe, dims, X)
    assert row_scaled_close(row_ptr, vals, host(s.vals)) <= VAL_TOL
    assert np.abs(host(s.b) - b).max() <= VAL_TOL * max(np.abs(b).max(), 1.0)


def test_rerun_is_bitwise_identical(fe):
    a = gpu_system(fe, (20, 20, 20))
    v1, b1 = host(a.vals), host(a.b)
    a.build()
    torch.cuda.synchronize()
    assert np.array_equal(v1, host(a.vals)) and np.array_equal(b1, host(a.b))


def oracle_row(dims, i):
    """Columns and values of row i, computed by the oracle one element at a time."""
    nx, ny, nz = dims
    nxn, nyn = nx + 1, ny + 1
    ix, iy, iz = i % nxn, (i // nxn) % nyn, i // (nxn * nyn)
    entries = {}
    for dz in (-1, 0):
        for dy in (-1, 0):
            for dx in (-1, 0):
                ex, ey, ez = ix + dx, iy + dy, iz + dz
                if not (0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz):
                    continue
                e = ex + nx * (ey + ny * ez)
                nodes = oracle.element_nodes(nx, ny, nz, e)
                X = np.array([[n % nxn / nx, (n // nxn) % nyn / ny, n // (nxn * nyn) / nz]
                              for n in nodes])
                K = oracle.element_matrix(X)
                a = int(np.nonzero(nodes == i)[0][0])
                for bb in range(8):
                    entries[int(nodes[bb])] = entries.get(int(nodes[bb]), 0.0) + K[a, bb]
    cols = sorted(entries)
    return np.array(cols), np.array([entries[c] for c in cols])


@pytest.mark.slow
def test_full_size_n256_sampled_rows(fe):
    """N = 256 (the benchmark's mesh): sampled interior rows against the oracle's
    element-by-element sums; boundary rows are identity rows."""
    dims = (256, 256, 256)
    s = gpu_system(fe, dims)
    m = s.m
    assert int(s.row_ptr[-1]) == (3 * 256 + 1) ** 3
    g = np.random.default_rng(0)
    rows = np.concatenate([[0, m - 1, m // 2], g.integers(0, m, size=60)])
    rp = host(s.row_ptr[torch.from_numpy(np.concatenate([rows, rows + 1])).cuda().long()])
    lo, hi = rp[:rows.size], rp[rows.size:]
    n = 257

    def on_boundary(j):
        ix, iy, iz = j % n, (j // n) % n, j // (n * n)
        return (ix == 0) | (ix == n - 1) | (iy == 0) | (iy == n - 1) | (iz == 0) | (iz == n - 1)

    for i, a, b_ in zip(rows, lo, hi):
        cols = host(s.cols[a:b_])
        vals = host(s.vals[a:b_])
        ref_cols, ref_vals = oracle_row(dims, int(i))
        assert np.array_equal(cols, ref_cols)
        if on_boundary(int(i)):
            assert np.array_equal(vals, (ref_cols == i).astype(float))
        else:
            scale = np.abs(ref_vals).max()
            ref_vals = np.where(on_boundary(ref_cols), 0.0, ref_vals)   # eliminated columns
            assert np.abs(vals - ref_vals).max() <= VAL_TOL * scale


@pytest.mark.slow
def test_largest_mesh_int32_limit(fe):
    """N = 429, the largest mesh whose 27-point pattern fits int32 row pointers
    ((3*429+1)^3 = 2,136,719,872 stored entries, 0.5 % below 2^31): the last row
    pointer equals the closed form, sampled rows match the oracle, and the CSR
    and BCRS3 SpMVs agree on sampled rows with the oracle's row dot products."""
    n = 429
    dims = (n, n, n)
    s = gpu_system(fe, dims)
    m = s.m
    assert int(s.row_ptr[-1]) == (3 * n + 1) ** 3
    g = np.random.default_rng(2)
    rows = np.concatenate([[0, m - 1, m // 2 + 7], g.integers(0, m, size=12)])
    x = torch.from_numpy(g.uniform(-1.0, 1.0, m)).cuda()
    y_csr = torch.empty_like(x)
    fe.fe_spmv(s.matrix("csr").desc, x, y_csr)
    A3 = s.matrix("bcrs3", "f64")
    y_b3 = torch.empty_like(x)
    fe.fe_spmv(A3.desc, x, y_b3)
    nn = n + 1
    xh = x.cpu().numpy()
    for i in rows:
        i = int(i)
        a, b_ = int(s.row_ptr[i]), int(s.row_ptr[i + 1])
        cols = s.cols[a:b_].cpu().numpy()
        vals = s.vals[a:b_].cpu().numpy()
        ref_cols, ref_vals = oracle_row(dims, i)
        assert np.array_equal(cols, ref_cols)
        ix, iy, iz = i % nn, (i // nn) % nn, i // (nn * nn)
        if min(ix, iy, iz) == 0 or max(ix, iy, iz) == n:
            want = xh[i]
        else:
            cx, cy, cz = ref_cols % nn, (ref_cols // nn) % nn, ref_cols // (nn * nn)
            bnd = (np.minimum(np.minimum(cx, cy), cz) == 0) | (np.maximum(np.maximum(cx, cy), cz) == n)
            ref_vals = np.where(bnd, 0.0, ref_vals)
            assert np.abs(vals - ref_vals).max() <= VAL_TOL * np.abs(ref_vals).max()
            want = float(np.dot(vals, xh[cols]))
        bound = 32 * 2.0 ** -53 * float(np.abs(vals) @ np.abs(xh[cols])) + 1e-300
        assert abs(float(y_csr[i]) - want) <= bound
        assert abs(float(y_b3[i]) - want) <= bound
