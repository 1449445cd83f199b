"""Mixed-precision form (FP32 or BF16 matrix values, FP32 inner CG with FP32
accumulation, FP64 residual, refinement and global dot products) checked
against the FP64 oracle, through the C ABI.

Per-form tolerances (the mixed-precision reading of the design notes):
  * the oracle's true relative residual of the result <= 1.5e-10 (tol 1e-10):
    the mixed form stops on the same FP64 residual test as the FP64 form;
  * the forward-error bound that test implies for any solution,
    ||x - x*|| <= ||b - A x|| / lambda_min(A), lambda_min from the closed-form
    Dirichlet spectrum (tests/test_oracle_spectrum.py) -- the guarantee;
  * a regression guard, ||x - x*|| <= 20 ||x_oracle - x*|| + 1e-12 ||x*||
    (x* the oracle solved to 1e-14): at the same residual the mixed form
    leaves more of its error in low modes than FP64 CG, measured 1.8-8.8x the
    FP64 form's error on the 97^3 and 257^3 meshes, so the guard sits at about
    twice the largest measured ratio; it is not a property of the method;
  * solved to 1e-13, the result matches the oracle's 1e-13 solution to 1e-10
    (the FP64 path's criterion (iv), one decade tighter for the same reason).
"""
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


REF = {}


def reference(dims, face=None):
    key = (dims, None if face is None else face.tobytes())
    if key not in REF:
        sysm = oracle.build_system(*dims, face)
        x, it, rel, st = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                   tol=1e-10, maxit=5000)
        xs, _, _, _ = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                tol=1e-14, maxit=20000)
        REF[key] = (sysm, x, xs)
    return REF[key]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def assert_forward_error(sysm, x, x_star, dims):
    """||x - x*|| <= (||b - A x|| + ||b - A x*||) / lambda_min(A)."""
    lam_min, _ = oracle.dirichlet_extreme_eigenvalues(*dims)
    res = lambda v: np.linalg.norm(sysm["b"] - oracle.spmv_csr(sysm["row_ptr"], sysm["cols"],
                                                              sysm["vals"], v))
    assert np.linalg.norm(x - x_star) <= (res(x) + res(x_star)) / lam_min


MODES = {"reliable": 0, "restart": 1}
INNER_TOL = {("restart", "f32"): 1e-5, ("restart", "bf16"): 1e-3,
             ("reliable", "f32"): 0.1, ("reliable", "bf16"): 0.1}


def solve_mixed(fe, s, fmt, value, mode="reliable", tol=1e-10, inner_tol=None, max_outer=60,
                max_inner=5000, hi="csr"):
    A64 = s.matrix(hi, "f64")
    Alo = s.matrix(fmt, value)
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    work = fe.mixed_workspace(Alo)
    res = fe.fe_cg_solve_mixed(A64.desc, Alo.desc, s.b, x, tol, MODES[mode], max_outer,
                               inner_tol or INNER_TOL[(mode, value)], max_inner, work,
                               check=False)
    return x, res


@pytest.mark.parametrize("mode", ["reliable", "restart"])
@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("value", ["f32", "bf16"])
def test_mixed_matches_fp64_oracle(fe, mode, fmt, value):
    dims = (30, 30, 30)
    sysm, x_or, x_star = reference(dims)
    s = fe.System(*dims).build()
    x, res = solve_mixed(fe, s, fmt, value, mode)
    assert res.status == fe.FE_OK and res.relres <= 1e-10
    xg = x.cpu().numpy()
    tr = oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg)
    assert tr <= 1.5e-10
    assert rel(xg, x_star) <= 20.0 * rel(x_or, x_star) + 1e-12
    assert_forward_error(sysm, xg, x_star, dims)
    assert res.outer_iterations >= 1 and res.inner_iterations >= res.outer_iterations


@pytest.mark.parametrize("mode", ["reliable", "restart"])
@pytest.mark.parametrize("value", ["f32", "bf16"])
def test_mixed_tight_tolerance_matches_oracle(fe, mode, value):
    dims = (30, 30, 30)
    sysm = reference(dims)[0]
    x13, _, _, st = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], tol=1e-13,
                              maxit=5000)
    s = fe.System(*dims).build()
    x, res = solve_mixed(fe, s, "bcrs3", value, mode, tol=1e-13)
    assert res.status == fe.FE_OK and res.relres <= 1e-13
    assert rel(x.cpu().numpy(), x13) <= 1e-10


@pytest.mark.parametrize("hi", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("lo", ["csr", "sell", "bcrs3"])
def test_reliable_format_pairs(fe, hi, lo):
    """Every pairing of FP64 and FP32 formats (the CSR ones stage in shared memory)."""
    dims = (25, 21, 19)
    sysm, x_or, x_star = reference(dims)
    s = fe.System(*dims).build()
    x, res = solve_mixed(fe, s, lo, "f32", hi=hi)
    assert res.status == fe.FE_OK
    xg = x.cpu().numpy()
    assert oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg) <= 1.5e-10


@pytest.mark.parametrize("hi", ["csr", "sell", "bcrs3"])
def test_reliable_bf16_cubic_any_fp64_format(fe, hi):
    dims = (24, 24, 24)
    sysm, x_or, x_star = reference(dims)
    s = fe.System(*dims).build()
    x, res = solve_mixed(fe, s, "csr", "bf16", hi=hi)
    assert res.status == fe.FE_OK
    xg = x.cpu().numpy()
    assert oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg) <= 1.5e-10


def test_reliable_bf16_stalls_honestly_on_skewed_mesh(fe):
    """BF16 rounding on non-cubic elements is not a uniform scaling of the
    operator; at value error x condition number ~ 1 the refinement cannot
    converge.  The solve must stop early with MAXIT and report the true
    residual, never claim convergence."""
    dims = (25, 21, 19)
    sysm = reference(dims)[0]
    s = fe.System(*dims).build()
    x, res = solve_mixed(fe, s, "bcrs3", "bf16")
    if res.status == fe.FE_OK:
        pytest.skip("converged on this mesh")
    assert res.status == fe.FE_ERR_MAXIT and res.inner_iterations < 5000
    tr = oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], x.cpu().numpy())
    assert abs(tr - res.relres) <= 1e-3 * tr and tr > 1e-10


@pytest.mark.parametrize("mode", ["reliable", "restart"])
@pytest.mark.parametrize("value", ["f32", "bf16"])
def test_mixed_face_data(fe, mode, value):
    dims = (20, 16, 24)
    face = fe_inputs.face_data(3, 9, *dims)
    sysm, x_or, x_star = reference(dims, face)
    s = fe.System(*dims, face_vals=torch.from_numpy(face).cuda()).build()
    x, res = solve_mixed(fe, s, "bcrs3", value, mode)
    assert res.status == fe.FE_OK
    xg = x.cpu().numpy()
    assert oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg) <= 1.5e-10
    assert rel(xg, x_star) <= 20.0 * rel(x_or, x_star) + 1e-12
    assert_forward_error(sysm, xg, x_star, dims)


@pytest.mark.parametrize("mode", ["reliable", "restart"])
def test_mixed_edge_cases(fe, mode):
    s = fe.System(6, 5, 4).build()
    # b = 0 gives x = 0 without an inner step
    s.b.zero_()
    x, res = solve_mixed(fe, s, "bcrs3", "bf16", mode)
    assert res.status == fe.FE_OK and res.outer_iterations == 0 and torch.count_nonzero(x) == 0
    s.build()
    # one refinement step allowed: stops with MAXIT after it
    x, res = solve_mixed(fe, s, "csr", "bf16", mode, max_outer=1)
    assert res.status == fe.FE_ERR_MAXIT and res.outer_iterations == 1
    assert 0 < res.relres < 1.0
    # a tolerance FP32 arithmetic alone cannot reach: the FP64 refinement gets there
    x, res = solve_mixed(fe, s, "sell", "f32", mode, tol=1e-13)
    assert res.status == fe.FE_OK and res.relres <= 1e-13


def test_reliable_rejects_fp64_inner(fe):
    s = fe.System(4).build()
    A64 = s.matrix("csr", "f64")
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        fe.fe_cg_solve_mixed(A64.desc, A64.desc, s.b, x, 1e-10, 0, 10, 0.1, 100,
                             fe.mixed_workspace(A64))
    assert e.value.status == fe.FE_ERR_ARG


def test_reliable_step_count_near_fp64(fe):
    """Refinement steps keep the Krylov space: with FP32 values the FP32 step
    count stays within 20% of the FP64 solve's; with BF16 values (value error
    2^-9 re-injected at each refinement step) within 2x."""
    s = fe.System(40).build()
    A = s.matrix("bcrs3", "f64")
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    ref = fe.fe_cg_solve(A.desc, s.b, x, 1e-10, 5000, fe.cg_workspace(A))
    for value, factor in (("f32", 1.2), ("bf16", 2.0)):
        x, res = solve_mixed(fe, s, "bcrs3", value)
        assert res.status == fe.FE_OK
        assert res.inner_iterations <= factor * ref.iterations + 5, (value, res.inner_iterations, ref.iterations)


@pytest.mark.slow
def test_full_size_n400_mixed(fe):
    """N = 400 (64.5M rows, the mixed-precision configuration): sampled assembled
    rows against the oracle, then FP64 CG and the reliable mixed solver with
    FP32 and BF16 values (BCRS3), each to a true relative residual <= 1.5e-10
    (FP64 residual kernel, pinned against the oracle in test_gpu_cg.py).  The
    per-form bars of the mixed form: the forward-error bound every solution
    meeting its residual obeys, ||x - x*|| <= ||b - A x|| / lambda_min(A) with
    lambda_min from the closed-form Dirichlet spectrum (4.6e-7 at N = 400;
    kappa(A) = 2.2e6, the identity rows setting lambda_max = 1), applied to
    x* = the FP64 solve to 1e-13; and the regression guard ||x - x*|| <=
    20 ||x_fp64 - x*|| + 1e-12 ||x*||."""
    import torch
    from test_gpu_assembly import oracle_row
    n = 400
    s = fe.System(n).build()
    m = s.m
    g = np.random.default_rng(1)
    rows = g.integers(0, m, size=24)
    nn = n + 1
    for i in rows:
        a, b_ = int(s.row_ptr[int(i)]), int(s.row_ptr[int(i) + 1])
        cols = s.cols[a:b_].cpu().numpy()
        vals = s.vals[a:b_].cpu().numpy()
        ref_cols, ref_vals = oracle_row((n, n, n), int(i))
        assert np.array_equal(cols, ref_cols)
        ix, iy, iz = i % nn, (i // nn) % nn, i // (nn * nn)
        if min(ix, iy, iz) == 0 or max(ix, iy, iz) == n:
            assert np.array_equal(vals, (ref_cols == i).astype(float))
        else:
            cx, cy, cz = ref_cols % nn, (ref_cols // nn) % nn, ref_cols // (nn * nn)
            bnd = (np.minimum(np.minimum(cx, cy), cz) == 0) | (np.maximum(np.maximum(cx, cy), cz) == n)
            ref_vals = np.where(bnd, 0.0, ref_vals)
            assert np.abs(vals - ref_vals).max() <= 1e-14 * np.abs(ref_vals).max()
    A64 = s.matrix("bcrs3", "f64")
    rwork = fe.resid_workspace()
    cwork = fe.cg_workspace(A64)
    bnorm = float(torch.linalg.norm(s.b))
    lam_min, _ = oracle.dirichlet_extreme_eigenvalues(n, n, n)
    xs = torch.zeros(m, dtype=torch.float64, device="cuda")
    r = fe.fe_cg_solve(A64.desc, s.b, xs, 1e-13, 20000, cwork)
    rs = fe.fe_true_relres(A64.desc, s.b, xs, rwork) * bnorm
    x64 = torch.zeros(m, dtype=torch.float64, device="cuda")
    r = fe.fe_cg_solve(A64.desc, s.b, x64, 1e-10, 20000, cwork)
    tr64 = fe.fe_true_relres(A64.desc, s.b, x64, rwork)
    assert r.status == fe.FE_OK and tr64 <= 1.5e-10
    e64 = float(torch.linalg.norm(x64 - xs))
    assert e64 <= (tr64 * bnorm + rs) / lam_min
    for v in ("f32", "bf16"):
        Alo = s.matrix("bcrs3", v)
        xm = torch.zeros_like(x64)
        rm = fe.fe_cg_solve_mixed(A64.desc, Alo.desc, s.b, xm, 1e-10, fe.FE_MIXED_RELIABLE, 200, 0.1,
                                  20000, fe.mixed_workspace(Alo), check=False)
        assert rm.status == fe.FE_OK, v
        trm = fe.fe_true_relres(A64.desc, s.b, xm, rwork)
        assert trm <= 1.5e-10
        em = float(torch.linalg.norm(xm - xs))
        assert em <= (trm * bnorm + rs) / lam_min, v
        assert em <= 20.0 * e64 + 1e-12 * float(torch.linalg.norm(xs)), (v, em / e64)
        del Alo, xm


# ---------------------------------------------------------------------------
# The BCRS3 inner matrix streams through a shared-memory ring filled by bulk
# copies when its column and value arrays start on 16-byte boundaries, and
# through thread loads otherwise.  Both walk the slots in the same order, so
# the solves must agree bit for bit.

def _shifted(t: torch.Tensor) -> torch.Tensor:
    """A copy of t whose storage starts one element past a 16-byte boundary."""
    buf = torch.empty(t.numel() + 16, dtype=t.dtype, device=t.device)
    assert buf.data_ptr() % 16 == 0
    out = buf[1:1 + t.numel()]
    out.copy_(t)
    assert out.data_ptr() % 16 != 0
    return out


def _with_arrays(fe, dm, cols, vals):
    d = dm.desc
    return fe.fe_matrix(d.format, d.value_type, d.n_rows, d.n_cols, d.n_slices, d.n_stored, None,
                        d.d_slice_ptr, cols.data_ptr(), vals.data_ptr())


def _bcrs3_from_csr(fe, row_ptr, cols, vals, m, value):
    """BCRS3 copy (values rounded to `value`) of an FP64 CSR matrix on the device."""
    ns = (m + 31) // 32
    csr = fe.fe_matrix(fe.FE_FMT_CSR, fe.FE_VAL_F64, m, m, ns, int(cols.numel()), row_ptr.data_ptr(), None,
                       cols.data_ptr(), vals.data_ptr())
    sp = torch.empty(ns + 1, dtype=torch.int64, device="cuda")
    n_stored = fe.fe_sliced_plan(fe.FE_FMT_BCRS3, m, m, row_ptr, cols, sp)
    c = torch.empty(n_stored, dtype=torch.int32, device="cuda")
    v = torch.empty(3 * n_stored, dtype=fe.TORCH_VALUE[fe.VALUE_TYPES[value]], device="cuda")
    d = fe.fe_matrix(fe.FE_FMT_BCRS3, fe.VALUE_TYPES[value], m, m, ns, n_stored, None, sp.data_ptr(),
                     c.data_ptr(), v.data_ptr())
    fe.fe_convert(csr, d)
    return csr, fe.DeviceMatrix(d, {"slice_ptr": sp, "cols": c, "vals": v})


def _solve_pair(fe, A64_desc, lo, b, m):
    """Reliable mixed solves with the aligned and the shifted inner arrays."""
    shifted = (_shifted(lo.tensors["cols"]), _shifted(lo.tensors["vals"]))
    lo_u = _with_arrays(fe, lo, *shifted)
    work = fe.mixed_workspace(lo)
    out = []
    for desc in (lo.desc, lo_u):
        x = torch.zeros(m, dtype=torch.float64, device="cuda")
        res = fe.fe_cg_solve_mixed(A64_desc, desc, b, x, 1e-10, MODES["reliable"], 60, 0.1, 5000, work,
                                   check=False)
        out.append((x, res))
    return out


@pytest.mark.parametrize("value", ["f32", "bf16"])
def test_reliable_staged_and_thread_load_paths_agree(fe, value):
    """70^3 elements (357,911 rows, 11,185 slices): every warp walks several
    slices per pass, so the ring is refilled and its parity turns over."""
    s = fe.System(70).build()
    (xa, ra), (xb, rb) = _solve_pair(fe, s.matrix("bcrs3", "f64").desc, s.matrix("bcrs3", value), s.b, s.m)
    assert ra.status == fe.FE_OK and rb.status == fe.FE_OK
    assert ra.inner_iterations == rb.inner_iterations and ra.outer_iterations == rb.outer_iterations
    assert torch.equal(xa, xb)


@pytest.mark.parametrize("value", ["f32", "bf16"])
@pytest.mark.parametrize("reach", [4, 12])
def test_reliable_staged_wide_and_narrow_slices(fe, value, reach):
    """A symmetric, strictly diagonally dominant matrix with couplings i +- 7k,
    k = 1..reach: every entry its own BCRS3 slot, so interior slices are nine
    slots wide (reach 4) or 25 (reach 12, the slices the ring passes to the
    global-memory walk), and the rows near both ends are narrower.  300,007
    rows.  The aligned and shifted solves agree bit for bit and reach the
    FP64 residual test, checked on the host."""
    m = 300_007
    i = np.arange(m, dtype=np.int64)
    offs = np.concatenate([-7 * np.arange(reach, 0, -1), [0], 7 * np.arange(1, reach + 1)])
    rows, cols, vals = [], [], []
    for o in offs:
        j = i + o
        keep = (j >= 0) & (j < m)
        rows.append(i[keep])
        cols.append(j[keep])
        vals.append(np.full(keep.sum(), 4.0 * reach + 1.0 if o == 0 else -1.0))
    rows, cols, vals = (np.concatenate(a) for a in (rows, cols, vals))
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=m))])
    b = np.cos(0.001 * i)
    d_rp = torch.from_numpy(row_ptr.astype(np.int32)).cuda()
    d_c = torch.from_numpy(cols.astype(np.int32)).cuda()
    d_v = torch.from_numpy(vals).cuda()
    d_b = torch.from_numpy(b).cuda()
    csr, lo = _bcrs3_from_csr(fe, d_rp, d_c, d_v, m, value)
    (xa, ra), (xb, rb) = _solve_pair(fe, csr, lo, d_b, m)
    assert ra.status == fe.FE_OK and rb.status == fe.FE_OK
    assert ra.inner_iterations == rb.inner_iterations
    assert torch.equal(xa, xb)
    x = xa.cpu().numpy()
    ax = np.bincount(rows, weights=vals * x[cols], minlength=m)
    assert np.linalg.norm(b - ax) <= 1.5e-10 * np.linalg.norm(b)
