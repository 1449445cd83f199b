"""The paper's BCRS on the GPU (Sec. 3.1, Fig 3.2/3.3: maximal runs of adjacent
columns, ptr / jas / offsets over the unchanged CRS values) against the
oracle, through the C ABI.

  * conversion: ptr, jas and offsets equal the oracle's (orc_csr_to_bcrs) bit
    for bit, including the length-6 runs of the one-element mesh;
  * SpMV: every value type, FP64 and FP32 vectors, element by element against
    the oracle's BCRS SpMV with the length-27 dot product's forward error
    bound (as test_gpu_spmv.py), on meshes up to several slices per warp;
  * CG: the FP64 criteria of test_gpu_cg.py against the oracle, in the
    three-phase, two-phase and single-reduction kernels (stop step within the
    multi-slice spread of test_gpu_multislice.py on the larger mesh).
"""
import numpy as np
import pytest
import torch

import fe_inputs
import oracle

pytestmark = pytest.mark.gpu

K = 27
U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def fe():
    import paper_1505_08023_gb300.fe as fe_mod
    fe_mod.load()
    return fe_mod


SYS = {}


def system(fe, dims):
    if dims not in SYS:
        ref = oracle.build_system(*dims)
        ptr, jas, off = oracle.csr_to_bcrs(ref["row_ptr"], ref["cols"])
        SYS[dims] = (fe.System(*dims).build(), ref, (ptr, jas, off))
    return SYS[dims]


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (5, 4, 3), (30, 30, 30), (97, 61, 45)])
def test_conversion_equals_the_oracle(fe, dims):
    s, ref, (ptr, jas, off) = system(fe, dims)
    A = s.matrix("vbcrs", "f64")
    assert A.desc.n_stored == jas.size
    assert np.array_equal(A.tensors["seg_ptr"].cpu().numpy(), ptr)
    assert np.array_equal(A.tensors["jas"].cpu().numpy(), jas)
    assert np.array_equal(A.tensors["seg_offsets"].cpu().numpy(), off)
    assert A.tensors["vals"].data_ptr() == s.vals.data_ptr()      # the CRS values, unchanged


def rounded(vals, value):
    return {"f64": vals, "f32": oracle.round_to_f32(vals), "bf16": oracle.round_to_bf16(vals)}[value]


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 4, 3), (30, 30, 30), (64, 64, 64), (97, 61, 45)])
@pytest.mark.parametrize("value", ["f64", "f32", "bf16"])
def test_spmv_against_the_oracle(fe, dims, value):
    s, ref, (ptr, jas, off) = system(fe, dims)
    A = s.matrix("vbcrs", value)
    gv = A.tensors["vals"].double().cpu().numpy()
    v = rounded(ref["vals"], value)
    x = fe_inputs.random_vector(41, s.m)
    y = torch.empty(s.m, dtype=torch.float64, device="cuda")
    fe.fe_spmv(A.desc, torch.from_numpy(x).cuda(), y)
    want = oracle.spmv_bcrs(ptr, jas, off, v, x)
    absum = oracle.spmv_bcrs(ptr, jas, off, np.abs(v), np.abs(x))
    slack = oracle.spmv_bcrs(ptr, jas, off, np.abs(gv - v), np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - want) <= 2 * K * U64 * absum + slack + 1e-300)
    x32 = x.astype(np.float32)
    y32 = torch.empty(s.m, dtype=torch.float32, device="cuda")
    fe.fe_spmv_f32(A.desc, torch.from_numpy(x32).cuda(), y32)
    x64 = x32.astype(np.float64)
    want = oracle.spmv_bcrs(ptr, jas, off, v, x64)
    absum = oracle.spmv_bcrs(ptr, jas, off, np.abs(v), np.abs(x64))
    slack = oracle.spmv_bcrs(ptr, jas, off, np.abs(gv - v), np.abs(x64))
    err = np.abs(y32.cpu().numpy().astype(np.float64) - want)
    assert np.all(err <= 2 * (K + 2) * U32 * absum + slack + 1e-38)


REF = {}


def reference(dims, form, tol):
    key = (dims, form, tol)
    if key not in REF:
        ref = system_ref(dims)
        solver = oracle.cg if form != "single_reduction" else oracle.cg_sr
        x, it, _, st = solver(ref["row_ptr"], ref["cols"], ref["vals"], ref["b"], tol=tol, maxit=5000)
        assert st == oracle.CG_CONVERGED
        REF[key] = (x, it)
    return REF[key]


def system_ref(dims):
    return SYS[dims][1]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims", [(30, 30, 30), (17, 9, 23), (64, 64, 64)])
@pytest.mark.parametrize("form", ["three_phase", "two_phase", "single_reduction"])
def test_cg_against_the_oracle(fe, dims, form):
    s, ref, _ = system(fe, dims)
    A = s.matrix("vbcrs", "f64")
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    if form == "single_reduction":
        res = fe.fe_cg_solve_sr(A.desc, s.b, x, 1e-10, 5000, fe.sr_workspace(A))
    else:
        f = fe.FE_CG_THREE_PHASE if form == "three_phase" else fe.FE_CG_TWO_PHASE
        res = fe.fe_cg_solve_form(A.desc, s.b, x, 1e-10, 5000, f, fe.cg_workspace(A))
    assert res.status == fe.FE_OK and res.relres <= 1e-10
    x_or, k_or = reference(dims, form, 1e-10)
    spread = 1 if dims[0] <= 30 else 3
    assert abs(res.iterations - k_or) <= spread, (res.iterations, k_or)
    xs, _ = reference(dims, "three_phase", 1e-14)
    xg = x.cpu().numpy()
    assert rel(xg, xs) <= 2.0 * rel(x_or, xs) + 1e-12
    assert oracle.true_relres(ref["row_ptr"], ref["cols"], ref["vals"], ref["b"], xg) <= 1.5e-10


def test_two_phase_is_bitwise_three_phase_and_resident_refuses(fe):
    s, _, _ = system(fe, (30, 30, 30))
    A = s.matrix("vbcrs", "f64")
    out = []
    for f in (fe.FE_CG_THREE_PHASE, fe.FE_CG_TWO_PHASE):
        x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
        r = fe.fe_cg_solve_form(A.desc, s.b, x, 1e-10, 5000, f, fe.cg_workspace(A))
        out.append((x, r.iterations))
    assert out[0][1] == out[1][1] and torch.equal(out[0][0], out[1][0])
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        fe.fe_cg_solve_form(A.desc, s.b, x, 1e-10, 100, fe.FE_CG_RESIDENT, fe.cg_workspace(A))
    assert e.value.status == fe.FE_ERR_ARG
