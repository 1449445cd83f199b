"""FP64 numpy oracle of the warm-start network's layers.

TEST INFRASTRUCTURE ONLY (the tests import it; the GPU path never does).

A 3x3x3 layer in "gather" form (the same definition the GPU kernels state):
    out[co][u] = bias[co] + sum_ci sum_t W[ci][t][co] in[ci][src(u, t)]
tap t = 9 dz + 3 dy + dx, per axis src = u + d - 1 (mode "s1"), 2u + d - 1
("s2") or (u + 1 - d)/2 when that is an integer ("t2"); zero outside the input
grid.  The gradients are written from that definition directly: the data
gradient scatters dY back through the same (u, t) -> src map, the weight
gradient sums dY[co][u] in[ci][src(u, t)] over u.
"""
from __future__ import annotations

import numpy as np

MODES = ("s1", "s2", "t2")


def out_dims(mode: str, dims):
    d = np.asarray(dims)
    if mode == "s1":
        return tuple(int(v) for v in d)
    if mode == "s2":
        return tuple(int(v) for v in (d - 1) // 2 + 1)
    return tuple(int(v) for v in 2 * (d - 1) + 1)


def _src_axis(mode: str, u: np.ndarray, d: int):
    """Source index along one axis and whether it exists (before range checks)."""
    if mode == "s1":
        return u + d - 1, np.ones_like(u, dtype=bool)
    if mode == "s2":
        return 2 * u + d - 1, np.ones_like(u, dtype=bool)
    p = u + 1 - d
    return p // 2, (p % 2) == 0


def _taps(mode: str, dims_in, dims_out):
    """For each tap: (flat source index per output voxel, validity mask)."""
    Di, Hi, Wi = dims_in
    Do, Ho, Wo = dims_out
    uz, uy, ux = np.meshgrid(np.arange(Do), np.arange(Ho), np.arange(Wo), indexing="ij")
    out = []
    for t in range(27):
        dz, dy, dx = t // 9, (t // 3) % 3, t % 3
        sz, vz = _src_axis(mode, uz, dz)
        sy, vy = _src_axis(mode, uy, dy)
        sx, vx = _src_axis(mode, ux, dx)
        ok = vz & vy & vx & (sz >= 0) & (sz < Di) & (sy >= 0) & (sy < Hi) & (sx >= 0) & (sx < Wi)
        flat = np.where(ok, (sz * Hi + sy) * Wi + sx, 0)
        out.append((flat.ravel(), ok.ravel()))
    return out


def conv(mode: str, x: np.ndarray, W: np.ndarray, bias=None, relu=False) -> np.ndarray:
    """x [cin][D][H][W], W [cin][27][cout] -> [cout][Do][Ho][Wo] (FP64)."""
    cin = x.shape[0]
    cout = W.shape[2]
    dims_in = x.shape[1:]
    dims_out = out_dims(mode, dims_in)
    xf = x.reshape(cin, -1).astype(np.float64)
    y = np.zeros((cout, int(np.prod(dims_out))))
    for t, (flat, ok) in enumerate(_taps(mode, dims_in, dims_out)):
        g = np.where(ok[None, :], xf[:, flat], 0.0)          # [cin][voxels]
        y += W[:, t, :].astype(np.float64).T @ g
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)[:, None]
    if relu:
        y = np.maximum(y, 0.0)
    return y.reshape((cout,) + dims_out)


def conv_grad_x(mode: str, dy: np.ndarray, W: np.ndarray, dims_in) -> np.ndarray:
    """d(loss)/dx for loss depending on y = conv(mode, x, W) (no ReLU)."""
    cin, cout = W.shape[0], W.shape[2]
    dims_out = dy.shape[1:]
    dyf = dy.reshape(cout, -1).astype(np.float64)
    dx = np.zeros((cin, int(np.prod(dims_in))))
    for t, (flat, ok) in enumerate(_taps(mode, dims_in, dims_out)):
        contrib = W[:, t, :].astype(np.float64) @ dyf       # [cin][voxels out]
        for ci in range(cin):
            np.add.at(dx[ci], flat[ok], contrib[ci][ok])
    return dx.reshape((cin,) + tuple(dims_in))


def conv_grad_w(mode: str, x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """d(loss)/dW [cin][27][cout] for y = conv(mode, x, W)."""
    cin, cout = x.shape[0], dy.shape[0]
    dims_in, dims_out = x.shape[1:], dy.shape[1:]
    xf = x.reshape(cin, -1).astype(np.float64)
    dyf = dy.reshape(cout, -1).astype(np.float64)
    dW = np.zeros((cin, 27, cout))
    for t, (flat, ok) in enumerate(_taps(mode, dims_in, dims_out)):
        g = np.where(ok[None, :], xf[:, flat], 0.0)
        dW[:, t, :] = g @ dyf.T
    return dW


def head(h: np.ndarray, w: np.ndarray, b: float) -> np.ndarray:
    """1x1x1 head: out[u] = b + sum_c w[c] h[c][u]."""
    return b + np.tensordot(np.asarray(w, dtype=np.float64), h.astype(np.float64), axes=(0, 0))


# ----------------------------------------------------------------------------
# The warm-start encoder-decoder, composed from the layers above (FP64).
# Same topology as the GPU network: encoder e0 (s1), d1 (s2), e1 (s1), d2, e2,
# d3, e3; decoder s2 = relu(t2(e3) + e2), f2 = relu(s1(s2)), s1 = relu(t2(f2)
# + e1), f1, s0 = relu(t2(f1) + e0), f0; head 1x1.  Loss: mean squared error
# over interior nodes.  `params` maps layer name -> (W [cin][27][cout], b).
# ----------------------------------------------------------------------------

ENC = [("e0", "s1", "x", 0), ("d1", "s2", "e0", 1), ("e1", "s1", "d1", 1), ("d2", "s2", "e1", 2),
       ("e2", "s1", "d2", 2), ("d3", "s2", "e2", 3), ("e3", "s1", "d3", 3)]
DEC = [("u2", "e3", "e2", "s2", "f2"), ("u1", "f2", "e1", "s1", "f1"), ("u0", "f1", "e0", "s0", "f0")]


def unet_forward(params, x):
    a = {"x": x}
    for name, mode, src, _ in ENC:
        W, b = params[name]
        a[name] = conv(mode, a[src], W, b, relu=True)
    for up, src, skip, s, f in DEC:
        W, b = params[up]
        a[s] = np.maximum(conv("t2", a[src], W, b) + a[skip], 0.0)
        W, b = params[f]
        a[f] = conv("s1", a[s], W, b, relu=True)
    hw, hb = params["head"]
    a["pred"] = head(a["f0"], hw, hb)
    return a


def unet_loss_grad(params, x, target, interior):
    """Loss and gradients (dict like params) of the network (FP64)."""
    a = unet_forward(params, x)
    n = interior.sum()
    diff = np.where(interior, a["pred"] - target, 0.0)
    loss = float(np.sum(diff * diff) / n)
    dpred = 2.0 * diff / n
    g = {}
    hw, hb = params["head"]
    g["head"] = (np.tensordot(a["f0"], dpred, axes=([1, 2, 3], [0, 1, 2])), float(dpred.sum()))
    da = {"f0": np.asarray(hw)[:, None, None, None] * dpred[None]}

    def layer_back(name, mode, inp, out, dout):
        dout = np.where(a[out] > 0, dout, 0.0) if out is not None else dout
        W, b = params[name]
        g[name] = (conv_grad_w(mode, a[inp], dout), dout.reshape(dout.shape[0], -1).sum(axis=1))
        return conv_grad_x(mode, dout, W, a[inp].shape[1:])

    skip_grad = {}
    for up, src, skip, s, f in reversed(DEC):
        ds = layer_back(f, "s1", s, f, da[f])
        ds = np.where(a[s] > 0, ds, 0.0)            # relu of the sum
        skip_grad[skip] = ds
        da[src] = layer_back(up, "t2", src, None, ds) + da.get(src, 0.0)
    for name, mode, src, _ in reversed(ENC):
        dout = da[name] + skip_grad.get(name, 0.0)
        dx = layer_back(name, mode, src, name, dout)
        if src != "x":
            da[src] = da.get(src, 0.0) + dx
    return loss, g
