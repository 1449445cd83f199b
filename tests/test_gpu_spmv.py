"""GPU parity of SpMV (paper Fig 3.1 CRS, Fig 3.2/3.3 BCRS) in every storage
format and value type against the oracle's CRS SpMV, through the C ABI.

Tolerances come from the forward error bound of a length-k dot product
(Higham, Thm 3.5): |fl(sum) - sum| <= gamma_k sum |a_ij x_j|, gamma_k ~ k u.
Both sides round, so the bar is 2 k u sum |a_ij x_j| with k = 27 (longest
row) and u = 2^-53 for FP64 accumulation, 2^-24 for FP32 accumulation.
Values stored in FP32/BF16: the oracle rounds its own FP64 values; the GPU
rounds its own.  Wherever the two FP64 inputs agree bit for bit the rounded
values must too, elsewhere they may differ by the FP64 difference plus one
unit of the stored type (the FP64 values agree to 1e-14 of the row scale).  The SpMV bar
adds the measured effect of those value differences, sum |dv_ij| |x_j|.
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


CASES = {}


def system(fe, dims):
    if dims not in CASES:
        s = fe.System(*dims).build()
        CASES[dims] = (s, oracle.build_system(*dims))
    return CASES[dims]


def rounded(ref_vals, value):
    return {"f64": ref_vals, "f32": oracle.round_to_f32(ref_vals),
            "bf16": oracle.round_to_bf16(ref_vals)}[value]


def gpu_values(s, value):
    """The GPU's stored values (every format rounds the same FP64 array elementwise)."""
    return s.matrix("csr", value).tensors["vals"].double().cpu().numpy()


def value_slack(s, ref, value, x):
    dv = np.abs(gpu_values(s, value) - rounded(ref["vals"], value))
    return oracle.spmv_csr(ref["row_ptr"], ref["cols"], dv, np.abs(x))


DIMS = [(1, 1, 1), (2, 2, 2), (5, 4, 3), (30, 30, 30), (31, 7, 13)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("value", ["f64", "f32", "bf16"])
def test_spmv_f64_vectors(fe, dims, fmt, value):
    s, ref = system(fe, dims)
    A = s.matrix(fmt, value)
    v = rounded(ref["vals"], value)
    m = s.m
    x = fe_inputs.random_vector(17, m)
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    fe.fe_spmv(A.desc, torch.from_numpy(x).cuda(), y)
    got = y.cpu().numpy()
    want = oracle.spmv_csr(ref["row_ptr"], ref["cols"], v, x)
    absum = oracle.spmv_csr(ref["row_ptr"], ref["cols"], np.abs(v), np.abs(x))
    slack = value_slack(s, ref, value, x)
    assert np.all(np.abs(got - want) <= 2 * K * U64 * absum + slack + 1e-300)


@pytest.mark.parametrize("dims", [(5, 4, 3), (30, 30, 30)])
@pytest.mark.parametrize("fmt", ["csr", "sell", "bcrs3"])
@pytest.mark.parametrize("value", ["f64", "f32", "bf16"])
def test_spmv_f32_vectors(fe, dims, fmt, value):
    s, ref = system(fe, dims)
    A = s.matrix(fmt, value)
    v = rounded(ref["vals"], value)
    x32 = fe_inputs.random_vector(18, s.m).astype(np.float32)
    y = torch.empty(s.m, dtype=torch.float32, device="cuda")
    fe.fe_spmv_f32(A.desc, torch.from_numpy(x32).cuda(), y)
    got = y.cpu().numpy().astype(np.float64)
    x = x32.astype(np.float64)
    # FP64 values enter the FP32 product rounded to FP32: one more u per term
    want = oracle.spmv_csr(ref["row_ptr"], ref["cols"], v, x)
    absum = oracle.spmv_csr(ref["row_ptr"], ref["cols"], np.abs(v), np.abs(x))
    slack = value_slack(s, ref, value, x)
    assert np.all(np.abs(got - want) <= 2 * (K + 2) * U32 * absum + slack + 1e-38)


@pytest.mark.parametrize("value", ["f32", "bf16"])
@pytest.mark.parametrize("dims", [(30, 30, 30), (31, 7, 13)])
def test_rounded_values(fe, value, dims):
    s, ref = system(fe, dims)
    got = gpu_values(s, value)
    want = rounded(ref["vals"], value)
    v64 = s.vals.cpu().numpy()
    same_input = v64 == ref["vals"]
    assert np.array_equal(got[same_input], want[same_input])
    # elsewhere rounding moves each value by at most half a unit of the stored
    # type, so the results differ by at most |dv| + one unit
    bits = 8 if value == "bf16" else 24
    ulp = np.ldexp(1.0, np.frexp(np.maximum(np.abs(want), np.abs(got)))[1] - bits)
    bound = np.abs(v64 - ref["vals"]) + ulp
    assert np.all(np.abs(got - want)[~same_input] <= bound[~same_input])


@pytest.mark.parametrize("fmt", ["sell", "bcrs3"])
def test_sliced_layout_invariants(fe, fmt):
    """Slot counts and padding of the sliced copies (sizes the roofline uses)."""
    dims = (30, 30, 30)
    s, ref = system(fe, dims)
    A = s.matrix(fmt, "f64")
    sp = A.tensors["slice_ptr"].cpu().numpy()
    assert sp[0] == 0 and np.all(np.diff(sp) % 32 == 0)
    n = dims[0] + 1
    if fmt == "bcrs3":
        nns = n * (3 * n - 2) ** 2             # one segment per (row, y/z neighbour line)
        assert sp[-1] >= nns and sp[-1] <= 9 * 32 * s.sizes.n_slices
        cols = A.tensors["cols"].cpu().numpy()
        assert cols.min() >= 0 and cols.max() <= s.m - 3
    else:
        assert sp[-1] >= s.sizes.nnz and sp[-1] <= 27 * 32 * s.sizes.n_slices


def test_spmv_repeatable(fe):
    s, ref = system(fe, (30, 30, 30))
    A = s.matrix("bcrs3", "f64")
    x = torch.from_numpy(fe_inputs.random_vector(3, s.m)).cuda()
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    fe.fe_spmv(A.desc, x, y1)
    fe.fe_spmv(A.desc, x, y2)
    assert torch.equal(y1, y2)
