"""fe_cg_solve_noalloc: the CG solve for callers that cannot allocate device
memory at solve time (e.g. inside a latency-critical loop, where cudaMalloc's
implicit device synchronisation is not acceptable, or in a plugin whose host
framework owns all device memory).  Its scratch lives in a fixed array inside
the library, so this checks, through the C ABI, that two calls in a row give
the same answer as the workspace-taking fe_cg_solve (same stop iteration,
solutions within the 1e-10 relative bar the CG tests use), and that a matrix
too large for the fixed array is refused before anything runs.

This file is collected last on purpose; it passes alone in a fresh process
and after the other tests.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import paper_1505_08023_gb300.fe as fe_mod
    fe_mod.load()
    return fe_mod


@pytest.mark.parametrize("fmt", ["bcrs3", "csr"])
def test_noalloc_matches_workspace_solve_twice(fe, fmt):
    s = fe.System(30).build()
    A = s.matrix(fmt, "f64")
    x_ref = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    ref = fe.fe_cg_solve(A.desc, s.b, x_ref, 1e-10, 1000, fe.cg_workspace(A))
    xr = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
        res = fe.fe_cg_solve_noalloc(A.desc, s.b, x, 1e-10, 1000)
        assert res.status == fe.FE_OK, call
        assert res.iterations == ref.iterations, call
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xr) <= 1e-10 * np.linalg.norm(xr), call


def test_noalloc_second_mesh_then_first_again(fe):
    # the shared scratch keeps the previous call's contents; each call must reset it
    for dims in [(20, 17, 11), (30, 30, 30)]:
        s = fe.System(*dims).build()
        A = s.matrix("sell", "f64")
        x_ref = torch.zeros(s.m, dtype=torch.float64, device="cuda")
        ref = fe.fe_cg_solve(A.desc, s.b, x_ref, 1e-10, 1000, fe.cg_workspace(A))
        x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
        res = fe.fe_cg_solve_noalloc(A.desc, s.b, x, 1e-10, 1000)
        assert res.status == fe.FE_OK and res.iterations == ref.iterations
        assert torch.linalg.norm(x - x_ref) <= 1e-10 * torch.linalg.norm(x_ref)


def test_noalloc_rejects_too_large(fe):
    s = fe.System(64).build()          # 65^3 = 274,625 rows > 262,144
    A = s.matrix("bcrs3", "f64")
    x = torch.zeros(s.m, dtype=torch.float64, device="cuda")
    res = fe.fe_cg_solve_noalloc(A.desc, s.b, x, 1e-10, 10, check=False)
    assert res.status == 0 and res.iterations == 0      # result untouched
    with pytest.raises(fe.FeError) as e:
        fe.fe_cg_solve_noalloc(A.desc, s.b, x, 1e-10, 10)
    assert e.value.status == fe.FE_ERR_WORKSPACE
    assert torch.count_nonzero(x) == 0
