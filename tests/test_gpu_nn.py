"""GPU kernels of the learned warm start against the FP64 network oracle
(oracle/nn.py), through the C ABI, and the warm start's effect on CG.

Both sides use the same BF16-rounded weights (the oracle applies them in
FP64).  FP32 accumulation of K products is bounded by 2 K 2^-24 sum |w||x|
(forward error of a dot product), written into each check.
"""
import numpy as np
import pytest
import torch

import fe_inputs
import oracle
from oracle import nn as onn

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def fe():
    import paper_1505_08023_gb300.fe as fe_mod
    fe_mod.load()
    return fe_mod


def bf16(a):
    return oracle.round_to_bf16(np.asarray(a, dtype=np.float32).astype(np.float64))


def cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


CASES = [("s1", 5, 20, (9, 7, 11)), ("s2", 17, 3, (9, 7, 11)), ("t2", 6, 16, (5, 4, 6)),
         ("s1", 2, 16, (17, 17, 17)), ("s2", 16, 32, (17, 17, 17)), ("t2", 64, 64, (3, 3, 3))]


def layer_setup(mode, cin, cout, dims, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal((cin,) + dims).astype(np.float32)
    W = bf16(0.2 * g.standard_normal((cin, 27, cout)))
    b = g.standard_normal(cout).astype(np.float32)
    return x, W, b


@pytest.mark.parametrize("mode,cin,cout,dims", CASES)
def test_conv_forward(fe, mode, cin, cout, dims):
    x, W, b = layer_setup(mode, cin, cout, dims, 1)
    dout = onn.out_dims(mode, dims)
    w32 = cuda32(W)
    w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(w32, cin, cout, 0, 0, w16)
    y = torch.empty((cout,) + dout, dtype=torch.float32, device="cuda")
    fe.fe_nn_conv3d(fe.NN_MODES[mode], cuda32(x), cin, dims, w16, cuda32(b), y, cout, dout, 0)
    ref = onn.conv(mode, x.astype(np.float64), W, b)
    bound = onn.conv(mode, np.abs(x).astype(np.float64), np.abs(W), np.abs(b))
    K = cin * 27 + 1
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 2 * K * U32 * bound + 1e-30)
    # fused ReLU
    fe.fe_nn_conv3d(fe.NN_MODES[mode], cuda32(x), cin, dims, w16, cuda32(b), y, cout, dout, 1)
    assert np.all(np.abs(y.cpu().numpy() - np.maximum(ref, 0)) <= 2 * K * U32 * bound + 1e-30)


@pytest.mark.parametrize("mode,cin,cout,dims", CASES)
def test_conv_data_gradient(fe, mode, cin, cout, dims):
    x, W, b = layer_setup(mode, cin, cout, dims, 2)
    dout = onn.out_dims(mode, dims)
    dy = np.random.default_rng(3).standard_normal((cout,) + dout).astype(np.float32)
    wt16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(cuda32(W), cin, cout, 1, 1 if mode == "s1" else 0, wt16)
    adj = {"s1": "s1", "s2": "t2", "t2": "s2"}[mode]
    dx = torch.empty((cin,) + dims, dtype=torch.float32, device="cuda")
    fe.fe_nn_conv3d(fe.NN_MODES[adj], cuda32(dy), cout, dout, wt16, None, dx, cin, dims, 0)
    ref = onn.conv_grad_x(mode, dy.astype(np.float64), W, dims)
    bound = onn.conv_grad_x(mode, np.abs(dy).astype(np.float64), np.abs(W), dims)
    K = cout * 27
    assert np.all(np.abs(dx.cpu().numpy() - ref) <= 2 * K * U32 * bound + 1e-30)


@pytest.mark.parametrize("mode,cin,cout,dims", CASES)
def test_conv_weight_gradient(fe, mode, cin, cout, dims):
    x, W, b = layer_setup(mode, cin, cout, dims, 4)
    dout = onn.out_dims(mode, dims)
    dy = np.random.default_rng(5).standard_normal((cout,) + dout).astype(np.float32)
    if mode == "t2":
        need, _ = fe.fe_nn_corr_workspace(2, cin, dims, cout)
    else:
        need, _ = fe.fe_nn_corr_workspace(1 if mode == "s1" else 2, cout, dout, cin)
    work = torch.empty(need // 4 + 1, dtype=torch.float32, device="cuda")
    dw = torch.empty((cin, 27, cout), dtype=torch.float32, device="cuda")
    fe.fe_nn_conv3d_weight_grad(fe.NN_MODES[mode], cuda32(x), cin, dims, cuda32(dy), cout, dout, dw, work)
    ref = onn.conv_grad_w(mode, x.astype(np.float64), dy.astype(np.float64))
    bound = onn.conv_grad_w(mode, np.abs(x).astype(np.float64), np.abs(dy).astype(np.float64))
    K = int(np.prod(dout)) if mode != "t2" else int(np.prod(dims))
    assert np.all(np.abs(dw.cpu().numpy() - ref) <= 2 * K * U32 * bound + 1e-30)
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    fe.fe_nn_channel_sum(cuda32(dy), cout, dout, db)
    assert np.allclose(db.cpu().numpy(), dy.reshape(cout, -1).astype(np.float64).sum(axis=1),
                       rtol=1e-5, atol=1e-4)


TC_CASES = [(2, 16, (9, 7, 11)), (16, 32, (17, 17, 17)), (32, 64, (5, 4, 6)), (64, 16, (3, 3, 3)),
            (16, 16, (4, 3, 129)), (20, 32, (6, 33, 65)), (16, 16, (1, 1, 1))]


@pytest.mark.parametrize("cin,cout,dims", TC_CASES)
def test_conv_s1_tensor_cores(fe, cin, cout, dims):
    """Stride-1 conv on tcgen05 against the FP64 oracle.  The kernel rounds
    activations to BF16 (relative error <= 2^-8 per product, nearest even)
    and accumulates in FP32, so |y - exact| <= (2^-8 + 2 K 2^-24) sum|w||x|.
    Cases cover partial 16-channel chunks, every allowed cout, grid widths
    of 129 and 65 (windows that straddle lines), and a single voxel."""
    x, W, b = layer_setup("s1", cin, cout, dims, 11)
    w32 = cuda32(W)
    w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(w32, cin, cout, 0, 0, w16)
    img = fe.mma_image(cin, cout)
    fe.fe_nn_pack_weights_mma(w16, cin, cout, img)
    bound = onn.conv("s1", np.abs(x).astype(np.float64), np.abs(W), np.abs(b))
    ref = onn.conv("s1", x.astype(np.float64), W, b)
    K = cin * 27 + 1
    tol = (2.0 ** -8 + 2 * K * U32) * bound + 1e-30
    y = torch.full((cout,) + dims, float("nan"), dtype=torch.float32, device="cuda")
    for relu in (0, 1):
        fe.fe_nn_conv3d_s1_tc(cuda32(x), cin, dims, img, cuda32(b), y, cout, relu)
        want = np.maximum(ref, 0) if relu else ref
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - want) <= tol), float(np.max(np.abs(got - want) / tol))
    assert fe.fe_nn_tc_check() == 0
    # the data-gradient copy (transposed, flipped taps) runs through the same kernel
    if cout in fe.TC_COUT and cin in fe.TC_COUT:
        dy = np.random.default_rng(12).standard_normal((cout,) + dims).astype(np.float32)
        wt16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
        fe.fe_nn_pack_weights(w32, cin, cout, 1, 1, wt16)
        imgt = fe.mma_image(cout, cin)
        fe.fe_nn_pack_weights_mma(wt16, cout, cin, imgt)
        dx = torch.empty((cin,) + dims, dtype=torch.float32, device="cuda")
        fe.fe_nn_conv3d_s1_tc(cuda32(dy), cout, dims, imgt, None, dx, cin, 0)
        refx = onn.conv_grad_x("s1", dy.astype(np.float64), W, dims)
        bx = onn.conv_grad_x("s1", np.abs(dy).astype(np.float64), np.abs(W), dims)
        tolx = (2.0 ** -8 + 2 * cout * 27 * U32) * bx + 1e-30
        assert np.all(np.abs(dx.cpu().numpy() - refx) <= tolx)


T2_TC_CASES = [(16, 16, (5, 4, 6)), (32, 16, (9, 9, 9)), (64, 64, (3, 3, 3)), (20, 32, (6, 17, 33)),
               (16, 32, (3, 5, 65)), (16, 16, (1, 1, 1))]


@pytest.mark.parametrize("cin,cout,dims", T2_TC_CASES)
def test_conv_t2_tensor_cores(fe, cin, cout, dims):
    """Transposed stride-2 conv on tcgen05 against the FP64 oracle, same BF16
    bound as the stride-1 kernel; also the stride-2 data gradient (the
    transposed layer with transposed weights) through the same kernel."""
    x, W, b = layer_setup("t2", cin, cout, dims, 13)
    dout = onn.out_dims("t2", dims)
    w32 = cuda32(W)
    w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(w32, cin, cout, 0, 0, w16)
    img = fe.mma_image(cin, cout)
    fe.fe_nn_pack_weights_mma(w16, cin, cout, img)
    ref = onn.conv("t2", x.astype(np.float64), W, b)
    bound = onn.conv("t2", np.abs(x).astype(np.float64), np.abs(W), np.abs(b))
    tol = (2.0 ** -8 + 2 * (cin * 27 + 1) * U32) * bound + 1e-30
    y = torch.full((cout,) + dout, float("nan"), dtype=torch.float32, device="cuda")
    for relu in (0, 1):
        fe.fe_nn_conv3d_t2_tc(cuda32(x), cin, dims, img, cuda32(b), y, cout, dout, relu)
        want = np.maximum(ref, 0) if relu else ref
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - want) <= tol), float(np.max(np.abs(got - want) / tol))
    assert fe.fe_nn_tc_check() == 0
    # data gradient of a stride-2 layer cin2 -> cout2 on the fine grid dout
    if cin in fe.TC_COUT:
        cin2, cout2 = cin, cout           # the stride-2 layer maps cin2 channels (fine) to cout2 (coarse)
        W2 = bf16(0.2 * np.random.default_rng(14).standard_normal((cin2, 27, cout2)))
        dy = np.random.default_rng(15).standard_normal((cout2,) + dims).astype(np.float32)
        wt16 = torch.empty(cin2 * 27 * cout2, dtype=torch.bfloat16, device="cuda")
        fe.fe_nn_pack_weights(cuda32(W2), cin2, cout2, 1, 0, wt16)
        imgt = fe.mma_image(cout2, cin2)
        fe.fe_nn_pack_weights_mma(wt16, cout2, cin2, imgt)
        dx = torch.empty((cin2,) + dout, dtype=torch.float32, device="cuda")
        fe.fe_nn_conv3d_t2_tc(cuda32(dy), cout2, dims, imgt, None, dx, cin2, dout, 0)
        refx = onn.conv_grad_x("s2", dy.astype(np.float64), W2, dout)
        bx = onn.conv_grad_x("s2", np.abs(dy).astype(np.float64), np.abs(W2), dout)
        tolx = (2.0 ** -8 + 2 * cout2 * 27 * U32) * bx + 1e-30
        assert np.all(np.abs(dx.cpu().numpy() - refx) <= tolx)


S2_TC_CASES = [(16, 32, (9, 7, 11)), (32, 64, (17, 17, 17)), (64, 64, (5, 5, 5)), (20, 16, (33, 9, 129)),
               (16, 16, (1, 1, 1)), (16, 16, (2, 3, 4))]


@pytest.mark.parametrize("cin,cout,dims", S2_TC_CASES)
def test_conv_s2_tensor_cores(fe, cin, cout, dims):
    """Stride-2 conv on tcgen05 (parity sub-box staging) against the FP64
    oracle, same BF16 bound; also the transposed layer's data gradient (the
    stride-2 layer with transposed weights) through the same kernel."""
    x, W, b = layer_setup("s2", cin, cout, dims, 16)
    dout = onn.out_dims("s2", dims)
    w32 = cuda32(W)
    w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(w32, cin, cout, 0, 0, w16)
    img = fe.mma_image(cin, cout)
    fe.fe_nn_pack_weights_mma(w16, cin, cout, img)
    ref = onn.conv("s2", x.astype(np.float64), W, b)
    bound = onn.conv("s2", np.abs(x).astype(np.float64), np.abs(W), np.abs(b))
    tol = (2.0 ** -8 + 2 * (cin * 27 + 1) * U32) * bound + 1e-30
    y = torch.full((cout,) + dout, float("nan"), dtype=torch.float32, device="cuda")
    for relu in (0, 1):
        fe.fe_nn_conv3d_s2_tc(cuda32(x), cin, dims, img, cuda32(b), y, cout, dout, relu)
        want = np.maximum(ref, 0) if relu else ref
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - want) <= tol), float(np.max(np.abs(got - want) / tol))
    assert fe.fe_nn_tc_check() == 0
    # data gradient of a transposed layer cin2 (coarse) -> cout2 (fine): dy on the fine grid
    if cin in fe.TC_COUT and all((d - 1) % 2 == 0 for d in dims):
        cin2, cout2 = cout, cin
        W2 = bf16(0.2 * np.random.default_rng(17).standard_normal((cin2, 27, cout2)))
        dy = np.random.default_rng(18).standard_normal((cout2,) + dims).astype(np.float32)
        wt16 = torch.empty(cin2 * 27 * cout2, dtype=torch.bfloat16, device="cuda")
        fe.fe_nn_pack_weights(cuda32(W2), cin2, cout2, 1, 0, wt16)
        imgt = fe.mma_image(cout2, cin2)
        fe.fe_nn_pack_weights_mma(wt16, cout2, cin2, imgt)
        dx = torch.empty((cin2,) + dout, dtype=torch.float32, device="cuda")
        fe.fe_nn_conv3d_s2_tc(cuda32(dy), cout2, dims, imgt, None, dx, cin2, dout, 0)
        refx = onn.conv_grad_x("t2", dy.astype(np.float64), W2, dout)
        bx = onn.conv_grad_x("t2", np.abs(dy).astype(np.float64), np.abs(W2), dout)
        tolx = (2.0 ** -8 + 2 * cout2 * 27 * U32) * bx + 1e-30
        assert np.all(np.abs(dx.cpu().numpy() - refx) <= tolx)


def test_conv_s1_tensor_cores_rejects_bad_cout(fe):
    x = torch.zeros((16, 3, 3, 3), device="cuda")
    img = fe.mma_image(16, 24)
    y = torch.zeros((24, 3, 3, 3), device="cuda")
    with pytest.raises(fe.FeError):
        fe.fe_nn_conv3d_s1_tc(x, 16, (3, 3, 3), img, None, y, 24, 0)


def test_network_gradients_match_oracle(fe):
    from paper_1505_08023_gb300 import warmstart as ws
    n = 9
    ch = (3, 4, 4, 5)
    g = np.random.default_rng(6)
    net = ws.WarmStartNet(n, channels=ch, tensor_cores=False)
    params = {}
    for name, l in net.layers.items():
        W = bf16(0.3 * g.standard_normal((l.cin, 27, l.cout)))
        b = (0.1 * g.standard_normal(l.cout)).astype(np.float32)
        l.w.copy_(cuda32(W))
        l.b.copy_(cuda32(b))
        params[name] = (W, b.astype(np.float64))
    hw = bf16(0.5 * g.standard_normal(ch[0]))
    net.hw.copy_(cuda32(hw))
    net.hb.fill_(0.05)
    params["head"] = (hw, float(np.float32(0.05)))
    net.pack()
    x = g.standard_normal((2, n, n, n)).astype(np.float32)
    target = g.standard_normal((n, n, n)).astype(np.float32)
    interior = np.zeros((n, n, n), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    flag = torch.from_numpy((~interior).astype(np.uint8).ravel()).cuda()
    pred = net.forward(cuda32(x))
    dpred = net.loss_and_grad(pred, cuda32(target), flag, int(interior.sum()))
    net.backward(dpred)
    loss_gpu = float(net.loss_parts.sum()) / interior.sum()
    loss, grad = onn.unet_loss_grad(params, x.astype(np.float64), target.astype(np.float64), interior)
    assert abs(loss_gpu - loss) <= 1e-4 * abs(loss)
    for name, l in net.layers.items():
        gw_ref, gb_ref = grad[name]
        gw = l.gw.cpu().numpy()
        assert np.linalg.norm(gw - gw_ref) <= 2e-4 * np.linalg.norm(gw_ref) + 1e-8, name
        assert np.linalg.norm(l.gb.cpu().numpy() - gb_ref) <= 2e-4 * np.linalg.norm(gb_ref) + 1e-8, name
    assert np.linalg.norm(net.ghw.cpu().numpy() - grad["head"][0]) <= 2e-4 * np.linalg.norm(grad["head"][0])


def test_adam_step(fe):
    g = np.random.default_rng(7)
    w, gr = g.standard_normal(1000).astype(np.float32), g.standard_normal(1000).astype(np.float32)
    m, v = np.zeros(1000, np.float32), np.zeros(1000, np.float32)
    tw, tg, tm, tv = cuda32(w), cuda32(gr), cuda32(m), cuda32(v)
    lr_t = 1e-3 * np.sqrt(1 - 0.999) / (1 - 0.9)
    fe.fe_nn_adam(tw, tg, tm, tv, lr_t, 0.9, 0.999, 1e-8)
    m1 = 0.1 * gr.astype(np.float64)
    v1 = 0.001 * gr.astype(np.float64) ** 2
    want = w - lr_t * m1 / (np.sqrt(v1) + 1e-8)
    assert np.allclose(tw.cpu().numpy(), want, rtol=1e-5, atol=1e-7)


def test_training_reduces_loss_and_warm_start_saves_iterations(fe):
    """N = 32: train on 96 CG solutions for 3 epochs, then solve 6 held-out
    problems from x0 = 0 and from the network's x0, each to 1e-10."""
    from paper_1505_08023_gb300 import warmstart as ws
    N = 32
    prob = ws.Problem(N)
    faces = ws.face_set(100, 0, 96, N)
    targets = ws.generate_targets(prob, faces)
    net = ws.WarmStartNet(N + 1, channels=(8, 16, 16, 16))
    log = ws.train(net, prob, faces, targets, epochs=3, lr=2e-3, log_every=24)
    first, last = log[0][2], log[-1][2]
    assert last < 0.5 * first
    rows = ws.evaluate(net, prob, ws.face_set(200, 0, 6, N))
    rep = ws.summarize(rows)
    assert rep["all_converged"]
    assert rep["mean_iters_warm"] < rep["mean_iters_cold"]
    assert rep["max_rel_diff_vs_cold"] < 1e-6
    # final error against the oracle on one held-out problem
    face = ws.face_set(200, 0, 1, N)[0]
    sysm = oracle.build_system(N, N, N, face)
    prob.set_faces(face)
    x0 = torch.empty(prob.sys.m, dtype=torch.float64, device="cuda")
    ws.predict_x0(net, prob, x0)
    r = fe.fe_cg_solve(prob.A.desc, prob.sys.b, x0, 1e-10, 5000, prob.work)
    tr = oracle.true_relres(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], x0.cpu().numpy())
    assert r.status == fe.FE_OK and tr <= 1.5e-10


def test_residual_loss_gradient(fe):
    """Problem.add_residual_grad adds (w / d^2) A (A dpred) with the FP32
    matrix; checked against the oracle's assembled CSR matrix in FP64."""
    from paper_1505_08023_gb300 import warmstart as ws
    N = 8
    prob = ws.Problem(N)
    face = ws.face_set(300, 0, 1, N)[0]
    prob.set_faces(face)
    sysm = oracle.build_system(N, N, N, face)
    g = np.random.default_rng(8)
    e = g.standard_normal(prob.sys.m)
    e[sysm["bc_flag"] != 0] = 0.0
    e = e.astype(np.float32)
    dpred = cuda32(e)
    prob.add_residual_grad(dpred, 0.5)
    rp, cols, vals = sysm["row_ptr"], sysm["cols"], sysm["vals"]
    A = lambda v: oracle.spmv_csr(rp, cols, vals, v)
    d = 8.0 / (3.0 * N)
    want = e.astype(np.float64) + 0.5 / d ** 2 * A(A(e.astype(np.float64)))
    got = dpred.cpu().numpy().astype(np.float64)
    assert np.all(got[sysm["bc_flag"] != 0] == 0.0)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("tc", [True, False])
def test_warmstart_infer_matches_layer_by_layer_forward(fe, tc):
    """fe_warmstart_infer (one C call) gives bit for bit the start vector of the
    layer-by-layer forward driven from Python, with and without tensor cores."""
    from paper_1505_08023_gb300 import warmstart as ws
    N = 16
    prob = ws.Problem(N)
    prob.set_faces(ws.face_set(400, 0, 1, N)[0])
    net = ws.WarmStartNet(N + 1, channels=(16, 16, 32, 32), tensor_cores=tc, seed=3)
    pred = net.forward(prob.x_in)
    want = torch.empty(prob.sys.m, dtype=torch.float64, device="cuda")
    fe.fe_warmstart_output(pred, prob.sys.bc_flag, prob.sys.bc_val, want)
    got = torch.full_like(want, float("nan"))
    ws.predict_x0(net, prob, got)
    assert torch.equal(got, want)
    assert fe.fe_nn_tc_check() == 0


def test_warmstart_infer_matches_oracle_network(fe):
    """fe_warmstart_infer on the CUDA-core path against the FP64 network oracle
    (same BF16 weights): interior values within 1e-4 of the largest |pred|,
    the compounded FP32 rounding of 14 layers; boundary values exact."""
    from paper_1505_08023_gb300 import warmstart as ws
    n = 9
    ch = (3, 4, 4, 5)
    prob = ws.Problem(n - 1)
    prob.set_faces(ws.face_set(401, 0, 1, n - 1)[0])
    g = np.random.default_rng(19)
    net = ws.WarmStartNet(n, channels=ch, tensor_cores=False)
    params = {}
    for name, l in net.layers.items():
        W = bf16(0.3 * g.standard_normal((l.cin, 27, l.cout)))
        b = (0.1 * g.standard_normal(l.cout)).astype(np.float32)
        l.w.copy_(cuda32(W))
        l.b.copy_(cuda32(b))
        params[name] = (W, b.astype(np.float64))
    hw = bf16(0.5 * g.standard_normal(ch[0]))
    net.hw.copy_(cuda32(hw))
    net.hb.fill_(0.05)
    params["head"] = (hw, float(np.float32(0.05)))
    net.pack()
    x0 = torch.empty(prob.sys.m, dtype=torch.float64, device="cuda")
    ws.predict_x0(net, prob, x0)
    flag = prob.sys.bc_flag.cpu().numpy().reshape((n,) * 3)
    val = prob.sys.bc_val.cpu().numpy().reshape((n,) * 3)
    xin = np.stack([np.where(flag != 0, val, 0.0), (flag != 0).astype(np.float64)])
    pred = onn.unet_forward(params, xin.astype(np.float32).astype(np.float64))["pred"]
    got = x0.cpu().numpy().reshape((n,) * 3)
    assert np.array_equal(got[flag != 0], val[flag != 0])
    inner = flag == 0
    assert np.max(np.abs(got[inner] - pred[inner])) <= 1e-4 * np.max(np.abs(pred))


def test_to_bf16i_layout(fe):
    """fe_nn_to_bf16i: [ceil(C/8)][V][8] BF16, nearest even, channels past C zero."""
    g = np.random.default_rng(20)
    c, dims = 11, (3, 4, 5)
    x = g.standard_normal((c,) + dims).astype(np.float32)
    buf = fe.bf16i_buffer(c, dims)
    fe.fe_nn_to_bf16i(cuda32(x), c, dims, buf)
    got = buf.view(torch.bfloat16).float().cpu().numpy().reshape(2, -1, 8)
    want = np.zeros((2, 60, 8))
    want[0] = bf16(x[:8].reshape(8, -1)).T
    want[1, :, :3] = bf16(x[8:].reshape(3, -1)).T
    assert np.array_equal(got, want)


TMA_CASES = [("s1", 16, 32, (9, 7, 11)), ("s1", 20, 16, (4, 3, 129)), ("s1", 64, 64, (5, 5, 5)),
             ("s2", 16, 32, (9, 7, 11)), ("s2", 20, 16, (33, 9, 129)), ("s2", 32, 64, (17, 17, 17)),
             ("t2", 16, 16, (5, 4, 6)), ("t2", 64, 32, (9, 9, 9)), ("t2", 16, 32, (3, 5, 65)),
             ("s1", 16, 16, (1, 1, 1)), ("s2", 16, 16, (2, 3, 4))]


@pytest.mark.parametrize("mode,cin,cout,dims", TMA_CASES)
def test_conv_tensor_cores_tma_staging(fe, mode, cin, cout, dims):
    """The TMA-staged tensor-core kernels (BF16 interleaved input) against the
    FP64 oracle with the BF16 bound, and bit for bit against the FP32-input
    tensor-core kernels (both round the same values to BF16 and run the same
    MMAs in the same order)."""
    x, W, b = layer_setup(mode, cin, cout, dims, 21)
    dout = onn.out_dims(mode, dims)
    w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    fe.fe_nn_pack_weights(cuda32(W), cin, cout, 0, 0, w16)
    img = fe.mma_image(cin, cout)
    fe.fe_nn_pack_weights_mma(w16, cin, cout, img)
    x16 = fe.bf16i_buffer(cin, dims)
    fe.fe_nn_to_bf16i(cuda32(x), cin, dims, x16)
    y = torch.full((cout,) + dout, float("nan"), dtype=torch.float32, device="cuda")
    fe.fe_nn_conv3d_tc_bf16i(mode, x16, cin, dims, img, cuda32(b), y, cout, dout, 1)
    ref = np.maximum(onn.conv(mode, x.astype(np.float64), W, b), 0)
    bound = onn.conv(mode, np.abs(x).astype(np.float64), np.abs(W), np.abs(b))
    tol = (2.0 ** -8 + 2 * (cin * 27 + 1) * U32) * bound + 1e-30
    got = y.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))
    y2 = torch.empty_like(y)
    fe.conv3d_tc(mode, cuda32(x), cin, dims, img, cuda32(b), y2, cout, dout, 1)
    assert torch.equal(y, y2)
    assert fe.fe_nn_tc_check() == 0


WG_TC_CASES = [("s1", 16, 20, (9, 7, 11)), ("s1", 32, 16, (17, 17, 17)), ("s1", 64, 64, (5, 6, 7)),
               ("s1", 16, 16, (1, 1, 1)), ("s1", 16, 16, (3, 5, 129)), ("s1", 16, 16, (33, 33, 33)),
               ("s2", 16, 32, (17, 17, 17)), ("s2", 64, 64, (9, 9, 9)), ("s2", 32, 8, (6, 10, 7)),
               ("t2", 32, 16, (5, 4, 6)), ("t2", 64, 32, (9, 9, 9)), ("t2", 16, 64, (3, 3, 3)),
               # grids too wide for a 256-point tensor-map box: B staged from FP32 by the threads
               ("s1", 16, 16, (2, 3, 260)), ("s2", 16, 16, (3, 3, 259))]


@pytest.mark.parametrize("mode,cin,cout,dims", WG_TC_CASES)
def test_conv_weight_gradient_tensor_cores(fe, mode, cin, cout, dims):
    """Weight gradient on tcgen05 (per tap a GEMM over the voxels, both operands
    rounded to BF16, FP32 accumulation, per-block partials summed in a fixed
    order) against the FP64 oracle: both operands are rounded to BF16 (8
    significant bits, relative error at most 2^-8 each), so each product's
    relative error is at most (1 + 2^-8)^2 - 1 = 2^-7 + 2^-16; the FP32 sums
    add 2 (K + splits) 2^-24, all times sum |x||dy|.  Covers one, two and four groups of taps (input
    channels of the correlation 16, 32, 64), the three layer kinds, and both
    ways of staging the second operand (tensor-map box loads of a BF16 copy;
    FP32 loads by the threads where the grid is too wide for the box)."""
    x, W, b = layer_setup(mode, cin, cout, dims, 6)
    dout = onn.out_dims(mode, dims)
    dy = np.random.default_rng(7).standard_normal((cout,) + dout).astype(np.float32)
    M = fe.NN_MODES[mode]
    need = fe.fe_nn_wgrad_tc_workspace(M, cin, dims, cout, dout)
    work = torch.empty(need // 4 + 1, dtype=torch.float32, device="cuda")
    dw = torch.empty((cin, 27, cout), dtype=torch.float32, device="cuda")
    fe.fe_nn_conv3d_weight_grad_tc(M, cuda32(x), cin, dims, cuda32(dy), cout, dout, dw, work)
    assert fe.fe_nn_tc_check() == 0
    ref = onn.conv_grad_w(mode, x.astype(np.float64), dy.astype(np.float64))
    bound = onn.conv_grad_w(mode, np.abs(x).astype(np.float64), np.abs(dy).astype(np.float64))
    K = int(np.prod(dout)) if mode != "t2" else int(np.prod(dims))
    splits = 256   # partials per weight: at most one per SM (152 on GB300), an upper bound
    tol = (2.0 ** -7 + 2.0 ** -16 + 2 * (K + splits) * U32) * bound
    assert np.all(np.abs(dw.cpu().numpy() - ref) <= tol + 1e-30)


def test_weight_gradient_tensor_cores_rejects_other_shapes(fe):
    # the correlation's N dimension (input channels for S1/S2, output for T2) must be 16, 32 or 64
    dims = (5, 5, 5)
    for mode, cin, cout in (("s1", 2, 16), ("s1", 24, 16), ("t2", 16, 8)):
        dout = onn.out_dims(mode, dims)
        with pytest.raises(fe.FeError) as e:
            fe.fe_nn_wgrad_tc_workspace(fe.NN_MODES[mode], cin, dims, cout, dout)
        assert e.value.status == fe.FE_ERR_ARG
