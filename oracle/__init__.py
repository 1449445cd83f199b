"""FP64 CPU oracle for the MiniFE heat-conduction path (arXiv 1505.08023).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package; the GPU library and its
Python binding never do.  It shares no code with the CUDA path.

The arithmetic lives in ``fe_oracle.c`` (plain serial C, compiled with
``-ffp-contract=off`` so each operation is one IEEE rounding on x86 and Arm);
this module compiles it on first use and wraps it with numpy arrays.  The
series solution the paper verifies against is in ``oracle.analytic``.

Parity pins (each checked by ``tests/test_oracle_*.py``):
  * element matrix       -- closed form (h/12)[4, 0, -1, -1] by the number of
                            differing corner coordinates; symmetric; zero row sums
  * pattern              -- nnz = (3nx+1)(3ny+1)(3nz+1), i.e. (3n-2)^3 with n
                            nodes per axis; row counts 27/18/12/8;
                            brute-force neighbour sets
  * assembled stencil    -- interior values 8h/3, 0, -h/6, -h/12; row sums 0
  * Dirichlet system     -- symmetric, Cholesky succeeds (SPD)
  * SpMV (CRS and BCRS)  -- dense matrix-vector product on small meshes
  * CG                   -- dense direct solve on meshes up to 4^3
  * single-reduction CG   -- Krylov termination (k distinct eigenvalues -> k
                            steps), textbook CG's iterates step by step,
                            dense direct solve, status codes
  * whole solve          -- series solution: centre value 1/6, O(h^2) error
  * matrix-free operator -- the assembled (element-integral) operator and
                            right-hand side on cubes and bricks; the closed-form
                            cube stencil; dense 1D Kronecker sums
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile fe_oracle.c into oracle/_build/liboracle.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_num_nodes.restype = i64
        lib.orc_num_nodes.argtypes = [i32, i32, i32]
        lib.orc_mesh.restype = None
        lib.orc_mesh.argtypes = [i32, i32, i32, ctypes.c_void_p, _f64p, _u8p, _f64p]
        lib.orc_element_matrix.restype = None
        lib.orc_element_matrix.argtypes = [_f64p, _f64p]
        lib.orc_element_nodes.restype = None
        lib.orc_element_nodes.argtypes = [i32, i32, i32, i64,
                                          np.ctypeslib.ndpointer(dtype=np.int64)]
        lib.orc_pattern.restype = i64
        lib.orc_pattern.argtypes = [i32, i32, i32, ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_assemble.restype = i32
        lib.orc_assemble.argtypes = [i32, i32, i32, _f64p, _i32p, _i32p, _f64p, _f64p]
        lib.orc_dirichlet.restype = None
        lib.orc_dirichlet.argtypes = [i64, _u8p, _f64p, _i32p, _i32p, _f64p, _f64p]
        lib.orc_spmv_csr.restype = None
        lib.orc_spmv_csr.argtypes = [i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.orc_csr_to_bcrs.restype = i64
        lib.orc_csr_to_bcrs.argtypes = [i64, _i32p, _i32p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_spmv_bcrs.restype = None
        lib.orc_spmv_bcrs.argtypes = [i64, _i32p, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.orc_dot.restype = f64
        lib.orc_dot.argtypes = [i64, _f64p, _f64p]
        lib.orc_cg.restype = i32
        lib.orc_cg.argtypes = [i64, _i32p, _i32p, _f64p, _f64p, _f64p, f64, i32,
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        lib.orc_cg_sr.restype = i32
        lib.orc_cg_sr.argtypes = lib.orc_cg.argtypes
        lib.orc_true_relres.restype = f64
        lib.orc_true_relres.argtypes = [i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.orc_stencil_coeffs.restype = None
        lib.orc_stencil_coeffs.argtypes = [i32, i32, i32, _f64p]
        lib.orc_stencil_row.restype = f64
        lib.orc_stencil_row.argtypes = [i32, i32, i32, i64, _f64p]
        lib.orc_stencil_spmv.restype = None
        lib.orc_stencil_spmv.argtypes = [i32, i32, i32, _f64p, _f64p]
        lib.orc_stencil_rhs.restype = None
        lib.orc_stencil_rhs.argtypes = [i32, i32, i32, _f64p, _f64p]
        _lib = lib
        return lib


# ----------------------------------------------------------------------------
# numpy-facing wrappers
# ----------------------------------------------------------------------------

def num_nodes(nx: int, ny: int, nz: int) -> int:
    return (nx + 1) * (ny + 1) * (nz + 1)


def face_sizes(nx: int, ny: int, nz: int) -> int:
    """Number of values in the concatenated face array (x0, x1, y0, y1, z0, z1)."""
    return 2 * ((ny + 1) * (nz + 1) + (nx + 1) * (nz + 1) + (nx + 1) * (ny + 1))


def mesh(nx: int, ny: int, nz: int, face_vals: np.ndarray | None = None):
    """Node coords (m, 3), boundary flags (m,) uint8 and boundary values (m,)."""
    lib = _load()
    m = num_nodes(nx, ny, nz)
    coords = np.empty((m, 3), dtype=np.float64)
    flag = np.empty(m, dtype=np.uint8)
    val = np.empty(m, dtype=np.float64)
    fv = None
    if face_vals is not None:
        fv = np.ascontiguousarray(face_vals, dtype=np.float64)
        if fv.size != face_sizes(nx, ny, nz):
            raise ValueError("face_vals has the wrong size")
    lib.orc_mesh(nx, ny, nz, None if fv is None else fv.ctypes.data, coords, flag, val)
    return coords, flag, val


def element_matrix(X: np.ndarray) -> np.ndarray:
    """8x8 element stiffness of the hexahedron with corner coordinates X (8, 3)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(24)
    K = np.empty(64, dtype=np.float64)
    lib.orc_element_matrix(X, K)
    return K.reshape(8, 8)


def element_nodes(nx: int, ny: int, nz: int, e: int) -> np.ndarray:
    lib = _load()
    out = np.empty(8, dtype=np.int64)
    lib.orc_element_nodes(nx, ny, nz, e, out)
    return out


def pattern(nx: int, ny: int, nz: int):
    """CRS row pointer and sorted columns of the 27-point pattern (Fig 3.6)."""
    lib = _load()
    nnz = lib.orc_pattern(nx, ny, nz, None, None)
    if nnz < 0:
        raise OverflowError("nnz does not fit an int32 row pointer")
    m = num_nodes(nx, ny, nz)
    row_ptr = np.empty(m + 1, dtype=np.int32)
    cols = np.empty(nnz, dtype=np.int32)
    lib.orc_pattern(nx, ny, nz, row_ptr.ctypes.data, cols.ctypes.data)
    return row_ptr, cols


def assemble(nx: int, ny: int, nz: int, coords, row_ptr, cols):
    """Global stiffness values (before boundary conditions) and zero RHS."""
    lib = _load()
    vals = np.empty(cols.shape[0], dtype=np.float64)
    b = np.empty(num_nodes(nx, ny, nz), dtype=np.float64)
    rc = lib.orc_assemble(nx, ny, nz, np.ascontiguousarray(coords), row_ptr, cols, vals, b)
    if rc != 0:
        raise RuntimeError("assembly met a column missing from the pattern")
    return vals, b


def dirichlet(bc_flag, bc_val, row_ptr, cols, vals, b):
    """Symmetric Dirichlet elimination in place (returns vals, b)."""
    lib = _load()
    lib.orc_dirichlet(bc_flag.shape[0], bc_flag, bc_val, row_ptr, cols, vals, b)
    return vals, b


def build_system(nx: int, ny: int, nz: int, face_vals=None):
    """Mesh -> pattern -> assembly -> Dirichlet: the full system A x = b."""
    coords, flag, gval = mesh(nx, ny, nz, face_vals)
    row_ptr, cols = pattern(nx, ny, nz)
    vals, b = assemble(nx, ny, nz, coords, row_ptr, cols)
    dirichlet(flag, gval, row_ptr, cols, vals, b)
    return dict(coords=coords, bc_flag=flag, bc_val=gval, row_ptr=row_ptr, cols=cols,
                vals=vals, b=b)


def spmv_csr(row_ptr, cols, vals, x):
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(row_ptr.shape[0] - 1, dtype=np.float64)
    lib.orc_spmv_csr(y.shape[0], row_ptr, cols, vals, x, y)
    return y


def csr_to_bcrs(row_ptr, cols):
    """The paper's variable-length BCRS index arrays: (ptr, jas, offsets)."""
    lib = _load()
    m = row_ptr.shape[0] - 1
    nns = lib.orc_csr_to_bcrs(m, row_ptr, cols, None, None, None)
    jas = np.empty(nns, dtype=np.int32)
    offsets = np.empty(nns + 1, dtype=np.int32)
    ptr = np.empty(m + 1, dtype=np.int32)
    lib.orc_csr_to_bcrs(m, row_ptr, cols, jas.ctypes.data, offsets.ctypes.data, ptr.ctypes.data)
    return ptr, jas, offsets


def spmv_bcrs(ptr, jas, offsets, vals, x):
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(ptr.shape[0] - 1, dtype=np.float64)
    lib.orc_spmv_bcrs(y.shape[0], ptr, jas, offsets, vals, x, y)
    return y


def dot(a, b) -> float:
    lib = _load()
    return lib.orc_dot(a.shape[0], np.ascontiguousarray(a, dtype=np.float64),
                       np.ascontiguousarray(b, dtype=np.float64))


CG_CONVERGED, CG_MAXIT, CG_BREAKDOWN = 0, 1, 2


def cg(row_ptr, cols, vals, b, x0=None, tol=1e-10, maxit=1000):
    """Textbook unpreconditioned CG; returns (x, iterations, relres, status)."""
    lib = _load()
    m = b.shape[0]
    x = np.zeros(m) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib.orc_cg(m, row_ptr, cols, vals, np.ascontiguousarray(b), x, float(tol),
                    int(maxit), ctypes.byref(it), ctypes.byref(rel))
    return x, it.value, rel.value, st


def cg_sr(row_ptr, cols, vals, b, x0=None, tol=1e-10, maxit=1000):
    """Single-reduction (Chronopoulos-Gear) CG; returns (x, iterations, relres, status)."""
    lib = _load()
    m = b.shape[0]
    x = np.zeros(m) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib.orc_cg_sr(m, row_ptr, cols, vals, np.ascontiguousarray(b), x, float(tol),
                       int(maxit), ctypes.byref(it), ctypes.byref(rel))
    return x, it.value, rel.value, st


def true_relres(row_ptr, cols, vals, b, x) -> float:
    lib = _load()
    return lib.orc_true_relres(b.shape[0], row_ptr, cols, vals, np.ascontiguousarray(b),
                               np.ascontiguousarray(x, dtype=np.float64))


def solve(nx: int, ny: int, nz: int, tol=1e-10, maxit=1000, face_vals=None, x0=None):
    """Whole path on the CPU: system assembly and CG.  Returns (system, x, iters, relres, status)."""
    sysm = build_system(nx, ny, nz, face_vals)
    x, it, rel, st = cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], x0, tol, maxit)
    return sysm, x, it, rel, st


# ----------------------------------------------------------------------------
# matrix-free form of the same system (Kronecker-sum stencil of the brick
# element; boundary rows identity, boundary columns eliminated)
# ----------------------------------------------------------------------------

def stencil_coeffs(nx: int, ny: int, nz: int) -> np.ndarray:
    """Interior stencil a[dz+1, dy+1, dx+1] of the assembled operator."""
    a = np.empty(27, dtype=np.float64)
    _load().orc_stencil_coeffs(nx, ny, nz, a)
    return a.reshape(3, 3, 3)


def stencil_spmv(nx: int, ny: int, nz: int, x) -> np.ndarray:
    """y = A x of the Dirichlet system without a stored matrix."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.shape[0] != num_nodes(nx, ny, nz):
        raise ValueError("x has the wrong length")
    y = np.empty_like(x)
    _load().orc_stencil_spmv(nx, ny, nz, x, y)
    return y


def stencil_row(nx: int, ny: int, nz: int, i: int, x) -> float:
    """(A x)_i for one row, matrix-free (for sampled checks on large meshes)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.shape[0] != num_nodes(nx, ny, nz) or not 0 <= i < x.shape[0]:
        raise ValueError("bad row or vector length")
    return _load().orc_stencil_row(nx, ny, nz, int(i), x)


def stencil_rhs(nx: int, ny: int, nz: int, bc_val) -> np.ndarray:
    """Right-hand side of the eliminated system from the boundary values."""
    g = np.ascontiguousarray(bc_val, dtype=np.float64)
    if g.shape[0] != num_nodes(nx, ny, nz):
        raise ValueError("bc_val has the wrong length")
    b = np.empty_like(g)
    _load().orc_stencil_rhs(nx, ny, nz, g, b)
    return b


def dirichlet_extreme_eigenvalues(nx: int, ny: int, nz: int):
    """(lambda_min, lambda_max) of the Dirichlet system A of the box mesh.

    Symmetric elimination (Sec. 1, boundary rows recorded by the mesh module)
    splits A into the identity on the boundary nodes and the interior block
    K_II.  On the brick mesh the trilinear element's stiffness is the Kronecker
    sum of 1D linear-element stiffness L = (1/h) tridiag(-1, 2, -1) and mass
    M = (h/6) tridiag(1, 4, 1), so K_II = Lx (x) My (x) Mz + Mx (x) Ly (x) Mz +
    Mx (x) My (x) Lz restricted to the interior nodes.  With Dirichlet ends the
    1D matrices share the eigenvectors sin(k pi j h), k = 1..N-1, with
    eigenvalues l(k) = (2/h)(1 - cos k pi h) and m(k) = (h/3)(2 + cos k pi h),
    and K_II's eigenvalues are lx(i) my(j) mz(k) + mx(i) ly(j) mz(k) +
    mx(i) my(j) lz(k).  The spectrum of A is that set together with 1.
    """
    def one_d(n):
        h = 1.0 / n
        k = np.arange(1, n, dtype=np.float64)
        c = np.cos(k * np.pi * h)
        return (2.0 / h) * (1.0 - c), (h / 3.0) * (2.0 + c)

    lo, hi = 1.0, 1.0                      # the boundary nodes' identity rows
    if min(nx, ny, nz) >= 2:
        lx, mx = one_d(nx)
        ly, my = one_d(ny)
        lz, mz = one_d(nz)
        lymz = np.multiply.outer(ly, mz)
        mylz = np.multiply.outer(my, lz)
        mymz = np.multiply.outer(my, mz)
        for i in range(lx.size):
            lam = lx[i] * mymz + mx[i] * (lymz + mylz)
            lo = min(lo, float(lam.min()))
            hi = max(hi, float(lam.max()))
    return lo, hi


def dense(row_ptr, cols, vals) -> np.ndarray:
    """Dense copy of a CRS matrix (small meshes only)."""
    m = row_ptr.shape[0] - 1
    A = np.zeros((m, m))
    for i in range(m):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            A[i, cols[k]] += vals[k]
    return A


# ----------------------------------------------------------------------------
# value rounding of the mixed-precision form (IEEE round to nearest, ties to
# even, directly from FP64); used to build the matrices the oracle multiplies
# when a GPU kernel stores its values in FP32 or BF16.
# ----------------------------------------------------------------------------

def round_to_f32(v: np.ndarray) -> np.ndarray:
    """FP64 values rounded to FP32 (nearest even), returned as FP64."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_to_bf16(v: np.ndarray) -> np.ndarray:
    """FP64 values rounded to bfloat16 (8-bit significand, nearest even), as FP64.

    Drops the low 45 of the 52 stored significand bits with round-half-even on
    the bit pattern; valid for finite values inside the bfloat16 normal range
    (every matrix value here is)."""
    bits = np.asarray(v, dtype=np.float64).view(np.uint64)
    drop = np.uint64(45)
    half = np.uint64((1 << 44) - 1)
    lsb = (bits >> drop) & np.uint64(1)
    rounded = (bits + half + lsb) & ~np.uint64((1 << 45) - 1)
    return rounded.view(np.float64)


# ----------------------------------------------------------------------------
# Multi-core CPU CG (fe_cpu_omp.c): a timing comparison for the benchmark's
# CPU leg, not part of the oracle's reference arithmetic.
# ----------------------------------------------------------------------------

_OMP_SRC = os.path.join(_HERE, "fe_cpu_omp.c")
_OMP_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_omp.so")
_omp_lib = None


def build_omp(force: bool = False) -> str:
    """Compile fe_cpu_omp.c into oracle/_build/liboracle_omp.so (gcc -O3 -fopenmp)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_OMP_LIB_PATH)
            and os.path.getmtime(_OMP_LIB_PATH) >= os.path.getmtime(_OMP_SRC)):
        return _OMP_LIB_PATH
    tmp = _OMP_LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _OMP_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OMP_LIB_PATH)
    return _OMP_LIB_PATH


def _load_omp():
    global _omp_lib
    with _lock:
        if _omp_lib is not None:
            return _omp_lib
        lib = ctypes.CDLL(build_omp())
        lib.omp_cg.restype = ctypes.c_int
        lib.omp_cg.argtypes = [ctypes.c_int64, ctypes.c_int, _i32p, _i32p, ctypes.c_void_p, _f64p,
                               _f64p, _f64p, ctypes.c_double, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        _omp_lib = lib
        return lib


def omp_cg(fmt: str, b, ptr, idx, vals, offsets=None, x0=None, tol=1e-10, maxit=1000):
    """Multi-core CG in CRS (fmt "csr": ptr = row_ptr, idx = cols) or the
    paper's BCRS (fmt "bcrs": ptr, idx = jas, offsets from csr_to_bcrs; vals =
    the CRS values).  Returns (x, iterations, relres, status, seconds, threads)."""
    lib = _load_omp()
    m = b.shape[0]
    x = np.zeros(m) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    f = {"csr": 0, "bcrs": 1}[fmt]
    if f == 1 and offsets is None:
        raise ValueError("BCRS needs offsets")
    off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int32)
    it, rel, sec, thr = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int(0)
    st = lib.omp_cg(m, f, ptr, idx, None if off is None else off.ctypes.data, vals,
                    np.ascontiguousarray(b), x, float(tol), int(maxit), ctypes.byref(it),
                    ctypes.byref(rel), ctypes.byref(sec), ctypes.byref(thr))
    return x, it.value, rel.value, st, sec.value, thr.value
