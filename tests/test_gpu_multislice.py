"""Oracle parity on the launch geometry the benchmark runs: meshes large enough
that every warp of the persistent kernels walks several 32-row slices and the
16-byte streaming passes take more than one trip per thread (the grid-stride
paths the N = 256 solve takes), compared element by element with the oracle.

SpMV (paper Fig 3.1 CRS, Fig 3.2/3.3 BCRS; sliced ELL): every format and value
type, bounded as in test_gpu_spmv.py (forward error of a length-27 dot
product, 2 k u sum |a_ij x_j|, plus the effect of stored-value differences).
CG (paper Sec. 1, textbook and single-reduction forms): the criteria of
test_gpu_cg.py -- the oracle's true residual of the GPU result <= 1.5e-10,
accuracy within 2x of the oracle's own against x* (the oracle solved to
1e-14), and solved to 1e-12 on both sides the two solutions within 1e-10 --
with the stop step within STOP_SPREAD of the oracle's.  On these meshes the
stop step itself moves with the summation order of the dot products: CPU runs
of the same recurrences with accurately summed dots in five orders (numpy's
pairwise dot, blocked sums of 64/1024/8192, exactly rounded) stop at 200-201
(textbook) and 199-202 (single reduction) on the 97^3 mesh, 134 and 134-135 on
the 65^3 mesh, so +-1 is not a property of CG there; +-3 is that spread.
"""
import numpy as np
import pytest
import torch

import fe_inputs
import oracle

pytestmark = pytest.mark.gpu

K = 27
U64, U32 = 2.0 ** -53, 2.0 ** -24
DIMS = [(64, 64, 64), (96, 96, 96), (97, 61, 45)]
THREADS, WARPS = 256, 8
STOP_SPREAD = 3


@pytest.fixture(scope="module")
def fe():
    import paper_1505_08023_gb300.fe as fe_mod
    fe_mod.load()
    return fe_mod


SYS = {}
REF = {}


def system(fe, dims):
    if dims not in SYS:
        SYS[dims] = (fe.System(*dims).build(), oracle.build_system(*dims))
    return SYS[dims]


def reference(dims, form, tol):
    key = (dims, form, tol)
    if key not in REF:
        ref = SYS[dims][1] if dims in SYS else oracle.build_system(*dims)
        solver = oracle.cg if form == "textbook" else oracle.cg_sr
        x, it, _, st = solver(ref["row_ptr"], ref["cols"], ref["vals"], ref["b"], tol=tol,
                              maxit=5000)
        assert st == oracle.CG_CONVERGED
        REF[key] = (x, it)
    return REF[key]


def x_star(dims):
    return reference(dims, "textbook", 1e-14)[0]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def resident_warps(blocks_per_sm):
    return torch.cuda.get_device_properties(0).multi_processor_count * blocks_per_sm * WARPS


@pytest.mark.parametrize("dims", DIMS)
def test_geometry_is_multi_slice(fe, dims):
    """The cases below really exercise the grid-stride paths: more slices than
    the persistent kernels' resident warps (4 blocks of 8 warps per SM at most),
    and at N = 96 more 16-byte vector packs than two per resident thread."""
    s, _ = system(fe, dims)
    assert s.sizes.n_slices > resident_warps(4)
    if dims == (96, 96, 96):
        packs = s.m // 2
        assert packs > 2 * torch.cuda.get_device_properties(0).multi_processor_count * 4 * THREADS


def rounded(vals, value):
    return {"f64": vals, "f32": oracle.round_to_f32(vals), "bf16": oracle.round_to_bf16(vals)}[value]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("value", ["f64", "f32", "bf16"])
def test_spmv_multi_slice(fe, dims, fmt, value):
    s, ref = system(fe, dims)
    A = s.matrix(fmt, value)
    v = rounded(ref["vals"], value)
    x = fe_inputs.random_vector(31, s.m)
    y = torch.empty(s.m, dtype=torch.float64, device="cuda")
    fe.fe_spmv(A.desc, torch.from_numpy(x).cuda(), y)
    got = y.cpu().numpy()
    want = oracle.spmv_csr(ref["row_ptr"], ref["cols"], v, x)
    absum = oracle.spmv_csr(ref["row_ptr"], ref["cols"], np.abs(v), np.abs(x))
    gv = s.matrix("csr", value).tensors["vals"].double().cpu().numpy()
    slack = oracle.spmv_csr(ref["row_ptr"], ref["cols"], np.abs(gv - v), np.abs(x))
    assert np.all(np.abs(got - want) <= 2 * K * U64 * absum + slack + 1e-300)
    if value != "f64":
        x32 = x.astype(np.float32)
        y32 = torch.empty(s.m, dtype=torch.float32, device="cuda")
        fe.fe_spmv_f32(A.desc, torch.from_numpy(x32).cuda(), y32)
        x64 = x32.astype(np.float64)
        want = oracle.spmv_csr(ref["row_ptr"], ref["cols"], v, x64)
        absum = oracle.spmv_csr(ref["row_ptr"], ref["cols"], np.abs(v), np.abs(x64))
        slack = oracle.spmv_csr(ref["row_ptr"], ref["cols"], np.abs(gv - v), np.abs(x64))
        err = np.abs(y32.cpu().numpy().astype(np.float64) - want)
        assert np.all(err <= 2 * (K + 2) * U32 * absum + slack + 1e-38)


def solve(fe, s, fmt, form, tol):
    A = s.matrix(fmt, "f64")
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    if form == "textbook":
        res = fe.fe_cg_solve(A.desc, s.b, x, tol, 5000, fe.cg_workspace(A))
    else:
        res = fe.fe_cg_solve_sr(A.desc, s.b, x, tol, 5000, fe.sr_workspace(A))
    assert res.status == fe.FE_OK and res.relres <= tol
    return x.cpu().numpy(), res.iterations


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("form", ["textbook", "single_reduction"])
def test_cg_multi_slice(fe, dims, fmt, form):
    s, ref = system(fe, dims)
    x_or, k_or = reference(dims, form, 1e-10)
    xg, kg = solve(fe, s, fmt, form, 1e-10)
    assert abs(kg - k_or) <= STOP_SPREAD, (kg, k_or)
    xs = x_star(dims)
    assert rel(xg, xs) <= 2.0 * rel(x_or, xs) + 1e-12
    tr = oracle.true_relres(ref["row_ptr"], ref["cols"], ref["vals"], ref["b"], xg)
    assert tr <= 1.5e-10, tr


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("form", ["textbook", "single_reduction"])
def test_cg_multi_slice_tight(fe, dims, form):
    """(iv): solved to 1e-12 on both sides the solutions agree to 1e-10 (BCRS3,
    the benchmark's format; the other formats share the CG kernel)."""
    s, _ = system(fe, dims)
    x_or, k_or = reference(dims, form, 1e-12)
    xg, kg = solve(fe, s, "bcrs3", form, 1e-12)
    assert abs(kg - k_or) <= STOP_SPREAD, (kg, k_or)
    assert rel(xg, x_or) <= 1e-10


# ---------------------------------------------------------------- mixed precision

def oracle_residual_norm(ref, x):
    r = ref["b"] - oracle.spmv_csr(ref["row_ptr"], ref["cols"], ref["vals"], x)
    return float(np.linalg.norm(r))


@pytest.mark.parametrize("value", ["f32", "bf16"])
@pytest.mark.parametrize("mode", ["reliable", "restart"])
def test_mixed_multi_slice(fe, value, mode):
    """Mixed form (FP32/BF16 values, FP32 inner CG, FP64 residual and
    refinement) on the N = 96 cube against the oracle, with the per-form bars:
    the oracle's true residual <= 1.5e-10; the forward-error bound every
    solution meeting that residual obeys, ||x - x*|| <= (||b - A x|| +
    ||b - A x*||) / lambda_min(A) (closed-form lambda_min); and the regression
    guard ||x - x*|| <= 20 ||x_oracle - x*|| + 1e-12 ||x*|| (the mixed-precision
    reading: about twice the largest measured ratio, 8.8)."""
    dims = (96, 96, 96)
    s, ref = system(fe, dims)
    x_or, _ = reference(dims, "textbook", 1e-10)
    xs = x_star(dims)
    A64, Alo = s.matrix("bcrs3", "f64"), s.matrix("bcrs3", value)
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    inner = {("restart", "f32"): 1e-5, ("restart", "bf16"): 1e-3}.get((mode, value), 0.1)
    res = fe.fe_cg_solve_mixed(A64.desc, Alo.desc, s.b, x, 1e-10,
                               fe.FE_MIXED_RELIABLE if mode == "reliable" else fe.FE_MIXED_RESTART,
                               100, inner, 20000, fe.mixed_workspace(Alo))
    assert res.status == fe.FE_OK
    xg = x.cpu().numpy()
    tr = oracle.true_relres(ref["row_ptr"], ref["cols"], ref["vals"], ref["b"], xg)
    assert tr <= 1.5e-10, tr
    lam_min, _ = oracle.dirichlet_extreme_eigenvalues(*dims)
    err = np.linalg.norm(xg - xs)
    assert err <= (oracle_residual_norm(ref, xg) + oracle_residual_norm(ref, xs)) / lam_min
    assert err <= 20.0 * np.linalg.norm(x_or - xs) + 1e-12 * np.linalg.norm(xs)
