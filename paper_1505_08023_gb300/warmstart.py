"""Learned warm start for the CG solve (an extension, not in the paper).

A 3-D convolutional encoder-decoder maps a mesh's boundary data (two input
channels on the (N+1)^3 node grid: boundary value, boundary flag) to a guess
of the solution at the interior nodes; the guess, with the prescribed values
on the boundary, is the CG start vector.  The FP64 solve still runs to the
same tolerance, so the network only changes how many steps it takes; when
the guess is worse than zero (||b - A x0|| > ||b||) the solve starts from 0.

Network (levels n, (n+1)/2, ... on the node grid; channels c0..c3):
    e0 = relu(S1(x))            c0       level 0
    d1 = relu(S2(e0))           c1       level 1       e1 = relu(S1(d1))
    d2 = relu(S2(e1))           c2       level 2       e2 = relu(S1(d2))
    d3 = relu(S2(e2))           c3       level 3       e3 = relu(S1(d3))
    s2 = relu(T2(e3) + e2)      f2 = relu(S1(s2))      level 2
    s1 = relu(T2(f2) + e1)      f1 = relu(S1(s1))      level 1
    s0 = relu(T2(f1) + e0)      f0 = relu(S1(s0))      level 0
    pred = head(f0)             1x1x1, one channel
Every layer runs in the project's kernels (fe_nn_*), BF16 weights and FP32
accumulation; training is Adam on FP32 master weights, loss = mean squared
error on interior nodes against FP64 CG solutions produced by this library's
batched solver.  Python only sequences the kernel calls and owns the tensors.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time

import numpy as np
import torch

from . import fe

CHANNELS = (16, 32, 64, 64)


def level_dims(n_nodes: int, levels: int = 4):
    if (n_nodes - 1) % (1 << (levels - 1)):
        raise ValueError("mesh size must be a multiple of 8 elements per axis")
    return [((n_nodes - 1) >> l) + 1 for l in range(levels)]


class Conv:
    """One 3x3x3 layer: FP32 master weights [cin][27][cout], bias, Adam moments,
    BF16 forward copy and BF16 copy for the data gradient; for stride-1 layers
    also their tensor-core operand images (when the output channel counts
    allow: 16, 32 or 64)."""

    def __init__(self, name, mode, cin, cout, dev, gen, tensor_cores=True):
        self.name, self.mode, self.cin, self.cout = name, mode, cin, cout
        fan_in = cin * 27
        std = math.sqrt(2.0 / fan_in)
        self.w = (torch.randn(cin, 27, cout, generator=gen, dtype=torch.float32) * std).to(dev)
        self.b = torch.zeros(cout, dtype=torch.float32, device=dev)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.w16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device=dev)
        self.wt16 = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device=dev)
        # tensor cores where both channel counts allow it: N (output channels)
        # 16, 32 or 64, and at least one full 16-channel K chunk (the 2-channel
        # input layer stays on the CUDA cores, where it is faster)
        # every mode runs forward and data gradient (its adjoint mode) on tcgen05
        fwd_tc = bwd_tc = tensor_cores
        self.img = fe.mma_image(cin, cout, dev) if fwd_tc and cout in fe.TC_COUT and cin >= 16 else None
        self.imgt = fe.mma_image(cout, cin, dev) if bwd_tc and cin in fe.TC_COUT and cout >= 16 else None

    def pack(self):
        fe.fe_nn_pack_weights(self.w, self.cin, self.cout, 0, 0, self.w16)
        flip = 1 if self.mode == "s1" else 0
        fe.fe_nn_pack_weights(self.w, self.cin, self.cout, 1, flip, self.wt16)
        if self.img is not None:
            fe.fe_nn_pack_weights_mma(self.w16, self.cin, self.cout, self.img)
        if self.imgt is not None:
            fe.fe_nn_pack_weights_mma(self.wt16, self.cout, self.cin, self.imgt)

    def params(self):
        return [(self.w, self.gw, self.mw, self.vw), (self.b, self.gb, self.mb, self.vb)]


ADJOINT = {"s1": "s1", "s2": "t2", "t2": "s2"}


class WarmStartNet:
    """The encoder-decoder.  tensor_cores=True runs every 3x3x3 layer with at
    least 16 input and 16/32/64 output channels (forward and data gradient)
    on tcgen05 with BF16 activations; False keeps every layer on the FP32
    CUDA-core kernels."""

    def __init__(self, n_nodes: int, channels=CHANNELS, device="cuda", seed: int = 0,
                 tensor_cores: bool = True):
        self.dev = torch.device(device)
        self.dims = [(d, d, d) for d in level_dims(n_nodes)]
        c0, c1, c2, c3 = channels
        self.ch = channels
        gen = torch.Generator().manual_seed(seed)
        L = lambda name, mode, ci, co: Conv(name, mode, ci, co, self.dev, gen, tensor_cores)
        self.layers = {
            "e0": L("e0", "s1", 2, c0), "d1": L("d1", "s2", c0, c1), "e1": L("e1", "s1", c1, c1),
            "d2": L("d2", "s2", c1, c2), "e2": L("e2", "s1", c2, c2), "d3": L("d3", "s2", c2, c3),
            "e3": L("e3", "s1", c3, c3), "u2": L("u2", "t2", c3, c2), "f2": L("f2", "s1", c2, c2),
            "u1": L("u1", "t2", c2, c1), "f1": L("f1", "s1", c1, c1), "u0": L("u0", "t2", c1, c0),
            "f0": L("f0", "s1", c0, c0)}
        self.hw = (torch.randn(c0, generator=gen) * math.sqrt(1.0 / c0)).float().to(self.dev)
        self.hb = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.ghw, self.ghb = torch.zeros_like(self.hw), torch.zeros_like(self.hb)
        self.mhw, self.vhw = torch.zeros_like(self.hw), torch.zeros_like(self.hw)
        self.mhb, self.vhb = torch.zeros_like(self.hb), torch.zeros_like(self.hb)
        self.hw16 = torch.empty(c0, dtype=torch.bfloat16, device=self.dev)
        self.step = 0
        self.tensor_cores = tensor_cores
        self.n_nodes = n_nodes
        self._blob = None
        self._infer_work = None
        self.buf = {}
        self.corr_work = None
        self.head_work = torch.empty((c0 + 1) * 64, dtype=torch.float32, device=self.dev)
        self.loss_parts = torch.empty(256, dtype=torch.float32, device=self.dev)
        self.pack()

    # ------------------------------------------------------------ helpers
    def pack(self):
        for l in self.layers.values():
            l.pack()
        self.hw16.copy_(self.hw.to(torch.bfloat16))
        self._blob = None            # the inference blob follows the weights

    def vol(self, key, c, level):
        d = self.dims[level]
        t = self.buf.get(key)
        if t is None or t.shape != (c,) + d:
            t = torch.empty((c,) + d, dtype=torch.float32, device=self.dev)
            self.buf[key] = t
        return t

    def bf16i(self, x, c, level):
        """x as BF16 8-channel-interleaved (the TMA-staged kernels' input)."""
        key = ("bf16i", c, level)
        buf = self.buf.get(key)
        if buf is None:
            buf = fe.bf16i_buffer(c, self.dims[level], self.dev)
            self.buf[key] = buf
        fe.fe_nn_to_bf16i(x, c, self.dims[level], buf)
        return buf

    def conv(self, lname, x, lin, y, lout, relu):
        l = self.layers[lname]
        if l.img is not None:
            x16 = self.bf16i(x, l.cin, lin)
            fe.fe_nn_conv3d_tc_bf16i(l.mode, x16, l.cin, self.dims[lin], l.img, l.b, y, l.cout, self.dims[lout],
                                     relu)
        else:
            fe.fe_nn_conv3d(fe.NN_MODES[l.mode], x, l.cin, self.dims[lin], l.w16, l.b, y, l.cout,
                            self.dims[lout], relu)

    def conv_bwd(self, lname, x, lin, dy, lout, dx):
        """Weight/bias gradients of layer lname; data gradient into dx (if given)."""
        l = self.layers[lname]
        stride = 1 if l.mode == "s1" else 2
        # the weight gradient on the tensor cores where the correlation's N
        # dimension (input channels; output channels of a transposed layer)
        # is 16, 32 or 64, else on the CUDA cores
        nb = l.cout if l.mode == "t2" else l.cin
        if self.tensor_cores and nb in (16, 32, 64):
            M = fe.NN_MODES[l.mode]
            need = fe.fe_nn_wgrad_tc_workspace(M, l.cin, self.dims[lin], l.cout, self.dims[lout])
            if self.corr_work is None or self.corr_work.numel() * 4 < need:
                self.corr_work = torch.empty(max(need // 4, 1) * 2, dtype=torch.float32, device=self.dev)
            fe.fe_nn_conv3d_weight_grad_tc(M, x, l.cin, self.dims[lin], dy, l.cout, self.dims[lout], l.gw,
                                           self.corr_work)
        else:
            if l.mode == "t2":
                need, _ = fe.fe_nn_corr_workspace(2, l.cin, self.dims[lin], l.cout)
            else:
                need, _ = fe.fe_nn_corr_workspace(stride, l.cout, self.dims[lout], l.cin)
            if self.corr_work is None or self.corr_work.numel() * 4 < need:
                self.corr_work = torch.empty(max(need // 4, 1) * 2, dtype=torch.float32, device=self.dev)
            fe.fe_nn_conv3d_weight_grad(fe.NN_MODES[l.mode], x, l.cin, self.dims[lin], dy, l.cout,
                                        self.dims[lout], l.gw, self.corr_work)
        fe.fe_nn_channel_sum(dy, l.cout, self.dims[lout], l.gb)
        if dx is not None:
            if l.imgt is not None:
                dy16 = self.bf16i(dy, l.cout, lout)
                fe.fe_nn_conv3d_tc_bf16i(ADJOINT[l.mode], dy16, l.cout, self.dims[lout], l.imgt, None, dx, l.cin,
                                         self.dims[lin], 0)
            else:
                fe.fe_nn_conv3d(fe.NN_MODES[ADJOINT[l.mode]], dy, l.cout, self.dims[lout], l.wt16, None,
                                dx, l.cin, self.dims[lin], 0)

    # ------------------------------------------------------------ forward / backward
    def forward(self, x):
        c0, c1, c2, c3 = self.ch
        V = self.vol
        e0 = V("e0", c0, 0); self.conv("e0", x, 0, e0, 0, 1)
        d1 = V("d1", c1, 1); self.conv("d1", e0, 0, d1, 1, 1)
        e1 = V("e1", c1, 1); self.conv("e1", d1, 1, e1, 1, 1)
        d2 = V("d2", c2, 2); self.conv("d2", e1, 1, d2, 2, 1)
        e2 = V("e2", c2, 2); self.conv("e2", d2, 2, e2, 2, 1)
        d3 = V("d3", c3, 3); self.conv("d3", e2, 2, d3, 3, 1)
        e3 = V("e3", c3, 3); self.conv("e3", d3, 3, e3, 3, 1)
        s2 = V("s2", c2, 2); self.conv("u2", e3, 3, s2, 2, 0)
        fe.fe_nn_axpy(1.0, e2, s2); fe.fe_nn_relu_bwd(s2, s2)
        f2 = V("f2", c2, 2); self.conv("f2", s2, 2, f2, 2, 1)
        s1 = V("s1", c1, 1); self.conv("u1", f2, 2, s1, 1, 0)
        fe.fe_nn_axpy(1.0, e1, s1); fe.fe_nn_relu_bwd(s1, s1)
        f1 = V("f1", c1, 1); self.conv("f1", s1, 1, f1, 1, 1)
        s0 = V("s0", c0, 0); self.conv("u0", f1, 1, s0, 0, 0)
        fe.fe_nn_axpy(1.0, e0, s0); fe.fe_nn_relu_bwd(s0, s0)
        f0 = V("f0", c0, 0); self.conv("f0", s0, 0, f0, 0, 1)
        pred = self.vol("pred", 1, 0)
        fe.fe_nn_head(f0, c0, self.dims[0], self.hw16, self.hb, pred)
        self.x_in = x
        return pred

    def backward(self, dpred):
        c0, c1, c2, c3 = self.ch
        B, V = self.buf, self.vol
        df0 = V("df0", c0, 0)
        fe.fe_nn_head_bwd(B["f0"], c0, self.dims[0], self.hw16, dpred, df0, self.ghw, self.ghb,
                          self.head_work)
        fe.fe_nn_relu_bwd(B["f0"], df0)
        ds0 = V("ds0", c0, 0); self.conv_bwd("f0", B["s0"], 0, df0, 0, ds0)
        fe.fe_nn_relu_bwd(B["s0"], ds0)                # grad of (u0 out + e0)
        df1 = V("df1", c1, 1); self.conv_bwd("u0", B["f1"], 1, ds0, 0, df1)
        fe.fe_nn_relu_bwd(B["f1"], df1)
        ds1 = V("ds1", c1, 1); self.conv_bwd("f1", B["s1"], 1, df1, 1, ds1)
        fe.fe_nn_relu_bwd(B["s1"], ds1)
        df2 = V("df2", c2, 2); self.conv_bwd("u1", B["f2"], 2, ds1, 1, df2)
        fe.fe_nn_relu_bwd(B["f2"], df2)
        ds2 = V("ds2", c2, 2); self.conv_bwd("f2", B["s2"], 2, df2, 2, ds2)
        fe.fe_nn_relu_bwd(B["s2"], ds2)
        de3 = V("de3", c3, 3); self.conv_bwd("u2", B["e3"], 3, ds2, 2, de3)
        fe.fe_nn_relu_bwd(B["e3"], de3)
        dd3 = V("dd3", c3, 3); self.conv_bwd("e3", B["d3"], 3, de3, 3, dd3)
        fe.fe_nn_relu_bwd(B["d3"], dd3)
        de2 = V("de2", c2, 2); self.conv_bwd("d3", B["e2"], 2, dd3, 3, de2)
        fe.fe_nn_axpy(1.0, ds2, de2)                   # skip into s2
        fe.fe_nn_relu_bwd(B["e2"], de2)
        dd2 = V("dd2", c2, 2); self.conv_bwd("e2", B["d2"], 2, de2, 2, dd2)
        fe.fe_nn_relu_bwd(B["d2"], dd2)
        de1 = V("de1", c1, 1); self.conv_bwd("d2", B["e1"], 1, dd2, 2, de1)
        fe.fe_nn_axpy(1.0, ds1, de1)                   # skip into s1
        fe.fe_nn_relu_bwd(B["e1"], de1)
        dd1 = V("dd1", c1, 1); self.conv_bwd("e1", B["d1"], 1, de1, 1, dd1)
        fe.fe_nn_relu_bwd(B["d1"], dd1)
        de0 = V("de0", c0, 0); self.conv_bwd("d1", B["e0"], 0, dd1, 1, de0)
        fe.fe_nn_axpy(1.0, ds0, de0)                   # skip into s0
        fe.fe_nn_relu_bwd(B["e0"], de0)
        self.conv_bwd("e0", self.x_in, 0, de0, 0, None)

    def all_params(self):
        out = []
        for l in self.layers.values():
            out += l.params()
        out += [(self.hw, self.ghw, self.mhw, self.vhw), (self.hb, self.ghb, self.mhb, self.vhb)]
        return out

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step += 1
        lr_t = lr * math.sqrt(1 - b2 ** self.step) / (1 - b1 ** self.step)
        for w, g, m, v in self.all_params():
            fe.fe_nn_adam(w, g, m, v, lr_t, b1, b2, eps)
        self.pack()

    def loss_and_grad(self, pred, target, bc_flag, n_interior):
        dpred = self.vol("dpred", 1, 0)
        fe.fe_nn_mse(pred, target, bc_flag, 1.0 / n_interior, dpred, self.loss_parts)
        return dpred

    def blob(self) -> torch.Tensor:
        """The weights as the fe_warmstart_infer blob (bias FP32 and BF16 weights
        per layer in the order e0 d1 e1 d2 e2 d3 e3 u2 f2 u1 f1 u0 f0, then the
        head), byte-for-byte the copies the layer kernels use."""
        offs, nbytes = fe.fe_warmstart_blob_layout(self.ch)
        out = torch.zeros(nbytes, dtype=torch.uint8, device=self.dev)
        order = ["e0", "d1", "e1", "d2", "e2", "d3", "e3", "u2", "f2", "u1", "f1", "u0", "f0"]
        for i, name in enumerate(order):
            l = self.layers[name]
            b = l.b.view(torch.uint8)
            out[offs[2 * i]:offs[2 * i] + b.numel()].copy_(b)
            w = l.w16.view(torch.uint8)
            out[offs[2 * i + 1]:offs[2 * i + 1] + w.numel()].copy_(w)
        hw = self.hw16.view(torch.uint8)
        out[offs[26]:offs[26] + hw.numel()].copy_(hw)
        hb = self.hb.view(torch.uint8)
        out[offs[27]:offs[27] + hb.numel()].copy_(hb)
        return out

    def state(self):
        d = {k: (l.w.cpu().numpy(), l.b.cpu().numpy()) for k, l in self.layers.items()}
        d["head"] = (self.hw.cpu().numpy(), self.hb.cpu().numpy())
        return d


# ---------------------------------------------------------------- data, training, evaluation

class Problem:
    """One mesh size: the shared matrix, mesh buffers reused per sample."""

    def __init__(self, N: int, device="cuda"):
        self.N = N
        self.dev = torch.device(device)
        self.sys = fe.System(N, device=self.dev)
        self.face = torch.empty(self.sys.sizes.n_faces, dtype=torch.float64, device=self.dev)
        self.sys.face_vals = self.face
        self.sys.build()
        self.A = self.sys.matrix("bcrs3", "f64")
        self.work = fe.cg_workspace(self.A, self.dev)
        self.x_in = torch.empty((2,) + (N + 1,) * 3, dtype=torch.float32, device=self.dev)
        self.n_interior = (N - 1) ** 3

    def set_faces(self, face_np, need_b: bool = True):
        self.face.copy_(torch.from_numpy(face_np))
        self.sys.generate_mesh()
        if need_b:
            self.sys.assemble()        # b for these faces (the matrix does not change)
        fe.fe_warmstart_input(self.sys.bc_flag, self.sys.bc_val, self.x_in)

    def add_residual_grad(self, dpred, weight: float):
        """Add the gradient of weight * sum((A e)^2) / (n d^2) to the MSE
        gradient dpred = 2 e / n, where e = pred - target is zero on boundary
        nodes and d = 8h/3 is the interior diagonal of A (so the term is
        dimensionless).  With q = A dpred = 2 A e / n and g = A q, that
        gradient is (weight / d^2) g; rows of boundary nodes are identity rows,
        so g stays zero there.  FP32 SELL SpMV."""
        if getattr(self, "A32", None) is None:
            self.A32 = self.sys.matrix("sell", "f32")
            self.q = torch.empty(self.sys.m, dtype=torch.float32, device=self.dev)
            self.g = torch.empty_like(self.q)
        flat = dpred.view(-1)
        fe.fe_spmv_f32(self.A32.desc, flat, self.q)
        fe.fe_spmv_f32(self.A32.desc, self.q, self.g)
        d = 8.0 / (3.0 * self.N)
        fe.fe_nn_axpy(weight / (d * d), self.g, flat)


def face_set(base_seed: int, first: int, count: int, N: int):
    import fe_inputs
    return [fe_inputs.face_data(base_seed, first + i, N, N, N) for i in range(count)]


def generate_targets(prob: Problem, faces, tol=1e-10, chunk=64):
    """FP64 CG solutions of the given boundary data (batched solver), stored in FP32."""
    N = prob.N
    out = torch.empty((len(faces),) + (N + 1,) * 3, dtype=torch.float32, device=prob.dev)
    for c0 in range(0, len(faces), chunk):
        sub = faces[c0:c0 + chunk]
        batch = fe.Batch([N] * len(sub), sub, "bcrs3", device=prob.dev)
        st, res = fe.fe_cg_solve_batched(batch.mats, batch.b, batch.x, tol, 20000, 4,
                                         batch.workspace())
        if st != fe.FE_OK:
            raise RuntimeError(f"batched solve failed: {fe.STATUS_NAMES.get(st, st)}")
        for i, x in enumerate(batch.x):
            out[c0 + i] = x.view((N + 1,) * 3).float()
        del batch
    return out


def train(net: WarmStartNet, prob: Problem, faces, targets, epochs=1, lr=1e-3, log_every=0,
          lr_final=None, res_weight=0.0):
    """Adam over the samples in a fixed shuffled order, one sample per step.
    With lr_final the step size follows a cosine from lr to lr_final; with
    res_weight > 0 the loss adds the scaled squared residual of the error
    (Problem.add_residual_grad), the quantity CG's stopping test measures."""
    losses = []
    n = len(faces)
    order = np.random.default_rng(0).permutation(n)
    total = epochs * n
    for ep in range(epochs):
        for k, i in enumerate(order):
            prob.set_faces(faces[i], need_b=False)
            pred = net.forward(prob.x_in)
            dpred = net.loss_and_grad(pred, targets[i], prob.sys.bc_flag, prob.n_interior)
            if res_weight > 0.0:
                prob.add_residual_grad(dpred, res_weight)
            net.backward(dpred)
            step_lr = lr
            if lr_final is not None:
                step_lr = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * (ep * n + k) / total))
            net.adam_step(step_lr)
            if log_every and (k % log_every == 0 or k == n - 1):
                losses.append((ep, k, float(net.loss_parts.sum()) / prob.n_interior))
    return losses


def predict_x0(net: WarmStartNet, prob: Problem, x0: torch.Tensor):
    """x0 from the mesh's boundary data: one fe_warmstart_infer call."""
    if net._blob is None:
        net._blob = net.blob()
    if net._infer_work is None:
        net._infer_work = fe._alloc_bytes(fe.fe_warmstart_workspace(net.n_nodes, net.ch), net.dev)
    fe.fe_warmstart_infer(net.n_nodes, net.ch, net._blob, prob.sys.bc_flag, prob.sys.bc_val, x0,
                          net._infer_work, net.tensor_cores)


BLOB_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT_BLOB = os.path.join(BLOB_DIR, "warmstart_n128.blob")


def save_blob(net: WarmStartNet, path: str, meta: dict):
    """Write the inference blob (the fe_warmstart_infer weight layout) and a
    JSON description of how it was trained beside it."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "wb") as f:
        f.write(net.blob().cpu().numpy().tobytes())
    info = dict(meta)
    info.update({"channels": list(net.ch), "n_nodes": net.n_nodes,
                 "layout": "fe_warmstart_blob_layout (bias FP32, weights BF16 per layer)"})
    with open(path + ".json", "w") as f:
        json.dump(info, f, indent=1)


class TrainedWarmStart:
    """Inference from a saved blob: x0 = network(boundary data), boundary
    nodes set to g exactly (one fe_warmstart_infer call)."""

    def __init__(self, path: str = DEFAULT_BLOB, device="cuda"):
        with open(path + ".json") as f:
            self.meta = json.load(f)
        self.ch = tuple(self.meta["channels"])
        self.n_nodes = int(self.meta["n_nodes"])
        raw = np.fromfile(path, dtype=np.uint8)
        _, nbytes = fe.fe_warmstart_blob_layout(self.ch)
        if raw.size != nbytes:
            raise ValueError(f"{path}: {raw.size} bytes, the layout of channels {self.ch} has {nbytes}")
        self.dev = torch.device(device)
        self.blob = torch.from_numpy(raw).to(self.dev)
        self.work = fe._alloc_bytes(fe.fe_warmstart_workspace(self.n_nodes, self.ch), self.dev)

    def predict(self, sys, x0: torch.Tensor, stream=None):
        if any(d + 1 != self.n_nodes for d in sys.dims):
            raise ValueError("the blob was trained for a different mesh")
        fe.fe_warmstart_infer(self.n_nodes, self.ch, self.blob, sys.bc_flag, sys.bc_val, x0, self.work,
                              True, stream)


def evaluate(net: WarmStartNet, prob: Problem, faces, tol=1e-10):
    """CG from x0 = 0 and from the network's x0 on each boundary data set."""
    EV = lambda: torch.cuda.Event(enable_timing=True)
    m = prob.sys.m
    x = torch.zeros(m, dtype=torch.float64, device=prob.dev)
    x0 = torch.empty_like(x)
    rwork = fe.resid_workspace(prob.dev)
    rows = []
    for f in faces:
        prob.set_faces(f)
        x.zero_()
        a, b = EV(), EV()
        a.record()
        r0 = fe.fe_cg_solve(prob.A.desc, prob.sys.b, x, tol, 20000, prob.work, check=False)
        b.record()
        torch.cuda.synchronize()
        t_cold = a.elapsed_time(b)
        x_cold = x.clone()
        a, b, c = EV(), EV(), EV()
        a.record()
        predict_x0(net, prob, x0)
        b.record()
        start_res = fe.fe_true_relres(prob.A.desc, prob.sys.b, x0, rwork)
        fallback = not (start_res < 1.0)
        if fallback:
            x0.zero_()
        r1 = fe.fe_cg_solve(prob.A.desc, prob.sys.b, x0, tol, 20000, prob.work, check=False)
        c.record()
        torch.cuda.synchronize()
        t_inf = a.elapsed_time(b)
        t_warm = a.elapsed_time(c)
        rows.append({"iters_cold": r0.iterations, "iters_warm": r1.iterations,
                     "ms_cold": t_cold, "ms_warm_incl_inference": t_warm, "ms_inference": t_inf,
                     "start_relres": start_res, "fallback": fallback,
                     "status_cold": r0.status, "status_warm": r1.status,
                     "relres_warm": r1.relres,
                     "rel_diff_vs_cold": float(torch.linalg.norm(x0 - x_cold) / torch.linalg.norm(x_cold))})
    return rows


def summarize(rows):
    ic = [r["iters_cold"] for r in rows]
    iw = [r["iters_warm"] for r in rows]
    tc = [r["ms_cold"] for r in rows]
    tw = [r["ms_warm_incl_inference"] for r in rows]
    return {"samples": len(rows), "mean_iters_cold": statistics.mean(ic),
            "mean_iters_warm": statistics.mean(iw),
            "iterations_saved_frac": 1.0 - statistics.mean(iw) / statistics.mean(ic),
            "mean_ms_cold": statistics.mean(tc), "mean_ms_warm_incl_inference": statistics.mean(tw),
            "time_saved_frac": 1.0 - statistics.mean(tw) / statistics.mean(tc),
            "mean_ms_inference": statistics.mean(r["ms_inference"] for r in rows),
            "mean_start_relres": statistics.mean(r["start_relres"] for r in rows),
            "fallbacks": sum(r["fallback"] for r in rows),
            "all_converged": all(r["status_warm"] == 0 and r["status_cold"] == 0 for r in rows),
            "max_rel_diff_vs_cold": max(r["rel_diff_vs_cold"] for r in rows)}


def run(N=128, n_train=2000, n_test=200, epochs=1, lr=1e-3, device="cuda", seed_train=1000,
        seed_test=2000, lr_final=None, res_weight=0.0, save=None):
    t0 = time.time()
    prob = Problem(N, device)
    faces_tr = face_set(seed_train, 0, n_train, N)
    faces_te = face_set(seed_test, 0, n_test, N)
    t1 = time.time()
    targets = generate_targets(prob, faces_tr)
    torch.cuda.synchronize()
    t2 = time.time()
    net = WarmStartNet(N + 1, device=device)
    losses = train(net, prob, faces_tr, targets, epochs=epochs, lr=lr, log_every=max(1, n_train // 10),
                   lr_final=lr_final, res_weight=res_weight)
    torch.cuda.synchronize()
    t3 = time.time()
    del targets
    if save:
        save_blob(net, save, {"N": N, "n_train": n_train, "epochs": epochs, "lr": lr,
                              "lr_final": lr_final, "res_weight": res_weight,
                              "train_seeds": f"PCG64({seed_train}, 0..{n_train - 1})",
                              "final_losses": losses[-3:] if losses else []})
    rows = evaluate(net, prob, faces_te)
    t4 = time.time()
    rep = summarize(rows)
    rep.update({"N": N, "n_train": n_train, "n_test": n_test, "epochs": epochs, "lr": lr,
                "lr_final": lr_final, "res_weight": res_weight,
                "train_seeds": f"PCG64({seed_train}, 0..{n_train - 1})",
                "test_seeds": f"PCG64({seed_test}, 0..{n_test - 1})",
                "s_faces": round(t1 - t0, 2), "s_targets": round(t2 - t1, 2),
                "s_train": round(t3 - t2, 2), "s_eval": round(t4 - t3, 2),
                "loss_log": losses})
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=None)
    ap.add_argument("--res-weight", type=float, default=0.0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-blob", default=None, help="write the trained inference blob here")
    a = ap.parse_args()
    rep = run(a.n, a.train, a.test, a.epochs, a.lr, lr_final=a.lr_final, res_weight=a.res_weight,
              save=a.save_blob)
    s = json.dumps(rep)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")


if __name__ == "__main__":
    main()
