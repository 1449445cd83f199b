"""Pins for the network oracle (oracle/nn.py): the stride-1 layer against
scipy's N-d correlation, the stride-2 and transposed layers against each
other (adjoint pair) and against brute force, gradients against finite
differences, and the shape rules of the 129 -> 65 -> 33 -> 17 ladder."""
import numpy as np
import pytest
import scipy.signal

from oracle import nn


def rand(g, *shape):
    return g.standard_normal(shape)


def test_s1_matches_scipy_correlate():
    g = np.random.default_rng(0)
    x = rand(g, 3, 5, 6, 7)
    W = rand(g, 3, 27, 2)
    y = nn.conv("s1", x, W)
    for co in range(2):
        ref = np.zeros(x.shape[1:])
        for ci in range(3):
            k = W[ci, :, co].reshape(3, 3, 3)
            ref += scipy.signal.correlate(x[ci], k, mode="same", method="direct")
        assert np.allclose(y[co], ref, atol=1e-12)


def test_s2_brute_force_and_shapes():
    g = np.random.default_rng(1)
    x = rand(g, 2, 7, 5, 9)
    W = rand(g, 2, 27, 3)
    y = nn.conv("s2", x, W)
    assert y.shape == (3, 4, 3, 5)
    for co, z, yy, xx in [(0, 0, 0, 0), (2, 3, 2, 4), (1, 2, 1, 3)]:
        s = 0.0
        for ci in range(2):
            for t in range(27):
                dz, dy, dx = t // 9, (t // 3) % 3, t % 3
                iz, iy, ix = 2 * z + dz - 1, 2 * yy + dy - 1, 2 * xx + dx - 1
                if 0 <= iz < 7 and 0 <= iy < 5 and 0 <= ix < 9:
                    s += W[ci, t, co] * x[ci, iz, iy, ix]
        assert abs(y[co, z, yy, xx] - s) < 1e-12
    assert nn.out_dims("s2", (129, 129, 129)) == (65, 65, 65)
    assert nn.out_dims("s2", (65, 65, 65)) == (33, 33, 33)
    assert nn.out_dims("t2", (17, 17, 17)) == (33, 33, 33)


def test_t2_is_adjoint_of_s2():
    g = np.random.default_rng(2)
    fine, coarse = (9, 7, 11), nn.out_dims("s2", (9, 7, 11))
    W = rand(g, 3, 27, 4)                       # s2: 3 -> 4 channels
    Wt = np.transpose(W, (2, 1, 0))             # t2: 4 -> 3 channels, W'[co][t][ci]
    x = rand(g, 3, *fine)
    z = rand(g, 4, *coarse)
    lhs = np.sum(nn.conv("s2", x, W) * z)
    rhs = np.sum(x * nn.conv("t2", z, Wt))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    assert nn.conv("t2", z, Wt).shape == (3,) + fine


@pytest.mark.parametrize("mode", nn.MODES)
def test_gradients_match_finite_differences(mode):
    g = np.random.default_rng(3)
    dims = (5, 4, 6) if mode != "t2" else (3, 3, 4)
    x = rand(g, 2, *dims)
    W = rand(g, 2, 27, 3)
    dims_out = nn.out_dims(mode, dims)
    c = rand(g, 3, *dims_out)                   # loss = sum(c * conv(x))

    def loss(xx, WW):
        return np.sum(c * nn.conv(mode, xx, WW))

    gx = nn.conv_grad_x(mode, c, W, dims)
    gW = nn.conv_grad_w(mode, x, c)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 1, 3), (0, dims[0] - 1, dims[1] - 1, dims[2] - 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (loss(xp, W) - loss(xm, W)) / (2 * eps)
        assert abs(fd - gx[idx]) < 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (1, 13, 2), (1, 26, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        fd = (loss(x, Wp) - loss(x, Wm)) / (2 * eps)
        assert abs(fd - gW[idx]) < 1e-6 * max(1.0, abs(fd))


def small_params(g, ch=(3, 4, 4, 5)):
    c0, c1, c2, c3 = ch
    shapes = {"e0": (2, c0), "d1": (c0, c1), "e1": (c1, c1), "d2": (c1, c2), "e2": (c2, c2),
              "d3": (c2, c3), "e3": (c3, c3), "u2": (c3, c2), "f2": (c2, c2), "u1": (c2, c1),
              "f1": (c1, c1), "u0": (c1, c0), "f0": (c0, c0)}
    p = {k: (0.3 * g.standard_normal((ci, 27, co)), 0.1 * g.standard_normal(co))
         for k, (ci, co) in shapes.items()}
    p["head"] = (0.5 * g.standard_normal(c0), 0.05)
    return p


def test_unet_gradient_matches_finite_differences():
    g = np.random.default_rng(5)
    n = 9                                           # levels 9, 5, 3, 2
    p = small_params(g)
    x = g.standard_normal((2, n, n, n))
    target = g.standard_normal((n, n, n))
    interior = np.zeros((n, n, n), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    loss, grad = nn.unet_loss_grad(p, x, target, interior)
    eps = 1e-6
    for name, idx in [("e0", (1, 13, 2)), ("d2", (0, 4, 3)), ("u2", (2, 26, 1)), ("f0", (0, 0, 0)),
                      ("e3", (4, 13, 4))]:
        W, b = p[name]
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        lp = nn.unet_loss_grad({**p, name: (Wp, b)}, x, target, interior)[0]
        lm = nn.unet_loss_grad({**p, name: (Wm, b)}, x, target, interior)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad[name][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, fd, grad[name][0][idx])
    W, b = p["e1"]
    bp = b.copy(); bp[1] += eps
    bm = b.copy(); bm[1] -= eps
    fd = (nn.unet_loss_grad({**p, "e1": (W, bp)}, x, target, interior)[0]
          - nn.unet_loss_grad({**p, "e1": (W, bm)}, x, target, interior)[0]) / (2 * eps)
    assert abs(fd - grad["e1"][1][1]) <= 1e-6 * max(1.0, abs(fd))
