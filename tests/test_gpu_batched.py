"""Batched form (many independent CG solves in one persistent launch) against
the CPU oracle, per system, through the C ABI.

Each system must meet the FP64 criteria of test_gpu_cg.py against its own
oracle solve: stop iteration within +-1, the oracle's true relative residual
<= 1.5e-10, and accuracy within 2x of the oracle's own at 1e-10.
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


def reference(n, face):
    key = (n, face.tobytes())
    if key not in REF:
        sysm = oracle.build_system(n, n, n, face)
        x, it, rel, st = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                   tol=1e-10, maxit=5000)
        xs, _, _, _ = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                tol=1e-14, maxit=20000)
        REF[key] = (sysm, it, x, xs)
    return REF[key]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SIZES = [6, 9, 6, 12, 9, 6, 15, 4]


def make_batch(fe, sizes, fmt, seed=0):
    faces = [fe_inputs.face_data(seed, i, n, n, n) for i, n in enumerate(sizes)]
    return fe.Batch(sizes, faces, fmt), faces


@pytest.mark.parametrize("fmt", ["bcrs3", "sell"])
@pytest.mark.parametrize("krhs", [1, 2, 4])
def test_batched_matches_oracle_per_system(fe, fmt, krhs):
    batch, faces = make_batch(fe, SIZES, fmt)
    st, res = fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, 1e-10, 2000, krhs,
                                     batch.workspace())
    assert st == fe.FE_OK
    for i, n in enumerate(SIZES):
        sysm, k_ref, x_or, x_star = reference(n, faces[i])
        assert res[i].status == fe.FE_OK
        assert abs(res[i].iterations - k_ref) <= 1, (i, res[i].iterations, k_ref)
        xg = batch.x[i].cpu().numpy()
        tr = oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], xg)
        assert tr <= 1.5e-10, (i, tr)
        assert rel(xg, x_star) <= 2.0 * rel(x_or, x_star) + 1e-12


def test_batched_matches_single_solves(fe):
    """Same systems through fe_cg_solve one by one: same stop rule, solutions
    within the 1e-10 bar of the CG tests (dot products are blocked differently)."""
    batch, faces = make_batch(fe, SIZES, "bcrs3", seed=3)
    st, res = fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, 1e-12, 2000, 2,
                                     batch.workspace())
    assert st == fe.FE_OK
    for i, n in enumerate(SIZES):
        A = batch.reps[n].matrix("bcrs3", "f64")
        x = torch.zeros_like(batch.x[i])
        r1 = fe.fe_cg_solve(A.desc, batch.b[i], x, 1e-12, 2000, fe.cg_workspace(A))
        assert abs(r1.iterations - res[i].iterations) <= 1
        assert torch.linalg.norm(x - batch.x[i]) <= 1e-10 * torch.linalg.norm(x)


def test_batched_bitwise_repeatable(fe):
    batch, _ = make_batch(fe, SIZES, "bcrs3", seed=4)
    work = batch.workspace()
    fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, 1e-10, 2000, 4, work)
    first = [x.clone() for x in batch.x]
    batch.reset()
    fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, 1e-10, 2000, 4, work)
    assert all(torch.equal(a, b) for a, b in zip(first, batch.x))


def test_batched_edge_cases(fe):
    sizes = [5, 7, 5]
    faces = [np.zeros(fe_inputs.face_data(0, 0, 5, 5, 5).size),
             fe_inputs.face_data(1, 1, 7, 7, 7), fe_inputs.face_data(1, 2, 5, 5, 5)]
    batch = fe.Batch(sizes, faces, "bcrs3")
    batch.x[0].fill_(3.0)
    st, res = fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, 1e-10, 2000, 2,
                                     batch.workspace())
    assert st == fe.FE_OK
    # zero boundary data: b = 0, x = 0 at once
    assert res[0].status == fe.FE_OK and res[0].iterations == 0
    assert torch.count_nonzero(batch.x[0]) == 0
    # maxit: every system stops at 3 steps with MAXIT
    batch.reset()
    st, res = fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, 1e-10, 3, 1, batch.workspace())
    assert st == fe.FE_ERR_MAXIT
    assert [r.status for r in res[1:]] == [fe.FE_ERR_MAXIT] * 2
    assert [r.iterations for r in res[1:]] == [3, 3]
    # one system alone
    one = fe.Batch([8], [fe_inputs.face_data(2, 0, 8, 8, 8)], "sell")
    st, res = fe.fe_cg_solve_batched(one.mats, one.b, one.x, 1e-10, 2000, 4, one.workspace())
    sysm, k_ref, _, _ = reference(8, fe_inputs.face_data(2, 0, 8, 8, 8))
    assert st == fe.FE_OK and abs(res[0].iterations - k_ref) <= 1


def test_batched_launch_replays_in_cuda_graph(fe):
    batch, faces = make_batch(fe, [10, 14, 10, 6], "bcrs3", seed=5)
    work = batch.workspace()
    plan = fe.fe_cg_batched_plan(batch.mats, batch.b, batch.x, 2, work)
    fe.fe_cg_batched_launch(plan, 1e-10, 2000)
    st, direct = fe.fe_cg_batched_results(plan)
    want = [x.clone() for x in batch.x]
    assert st == fe.FE_OK
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    batch.reset()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        for x in batch.x:
            x.zero_()
        fe.fe_cg_batched_launch(plan, 1e-10, 2000, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        st, res = fe.fe_cg_batched_results(plan)
        assert st == fe.FE_OK
        assert [r.iterations for r in res] == [r.iterations for r in direct]
        assert all(torch.equal(a, b) for a, b in zip(want, batch.x))


def test_batched_rejects_mixed_formats(fe):
    a = fe.Batch([4, 5], None, "bcrs3")
    b = fe.Batch([4], None, "sell")
    with pytest.raises(fe.FeError):
        fe.fe_cg_batched_plan([a.mats[0], b.mats[0]], [a.b[0], b.b[0]], [a.x[0], b.x[0]], 1,
                              a.workspace())


def test_autotuner_choice_solves(fe):
    from paper_1505_08023_gb300 import autotune
    batch, faces = make_batch(fe, [8, 12, 8, 10], "bcrs3", seed=7)
    choice = autotune.tune(batch, steps=8, repeats=1)
    assert choice.fmt in ("bcrs3", "sell") and choice.krhs in (1, 2, 4)
    assert autotune.tune(batch) is choice            # cached by signature
    mats = batch.mats_for(choice.fmt)
    st, res = fe.fe_cg_solve_batched(mats, batch.b, batch.x, 1e-10, 2000, choice.krhs,
                                     batch.workspace())
    assert st == fe.FE_OK
    for i, n in enumerate([8, 12, 8, 10]):
        sysm, k_ref, _, _ = reference(n, faces[i])
        assert abs(res[i].iterations - k_ref) <= 1
