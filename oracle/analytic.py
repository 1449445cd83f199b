"""Series solution of the paper's problem (Sec. 1: unit cube, T = 1 on x = 1,
T = 0 on the other faces), which the paper's verification module compares the
FE solution against.

TEST INFRASTRUCTURE ONLY (imported by the tests and nothing in the GPU path).

Separation of variables for Laplace's equation: the face value 1 has the sine
series 1 = sum_{m,n odd} 16/(pi^2 m n) sin(m pi y) sin(n pi z) on (0,1)^2, and
each term continues into the cube as sinh(g x)/sinh(g) with g = pi sqrt(m^2+n^2):

    T(x,y,z) = sum_{m,n odd} 16/(pi^2 m n) sin(m pi y) sin(n pi z) sinh(g x)/sinh(g).

The sinh ratio is evaluated in the overflow-free form
exp(g (x-1)) (1 - exp(-2 g x)) / (1 - exp(-2 g)).
"""
from __future__ import annotations

import numpy as np


def series(x, y, z, max_mode: int = 401, chunk: int = 4096) -> np.ndarray:
    """T at the points (x, y, z) (broadcast arrays) from odd modes m, n <= max_mode."""
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float),
                                  np.asarray(z, float))
    shape = x.shape
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    modes = np.arange(1, max_mode + 1, 2, dtype=float)
    mm, nn = np.meshgrid(modes, modes, indexing="ij")
    mm, nn = mm.ravel(), nn.ravel()
    gam = np.pi * np.sqrt(mm * mm + nn * nn)
    coef = 16.0 / (np.pi ** 2 * mm * nn)
    out = np.empty(x.shape[0])
    for s in range(0, x.shape[0], chunk):
        xs, ys, zs = x[s:s + chunk, None], y[s:s + chunk, None], z[s:s + chunk, None]
        ratio = np.exp(gam * (xs - 1.0)) * (1.0 - np.exp(-2.0 * gam * xs)) \
            / (1.0 - np.exp(-2.0 * gam))
        terms = coef * np.sin(mm * np.pi * ys) * np.sin(nn * np.pi * zs) * ratio
        out[s:s + chunk] = terms.sum(axis=1)
    return out.reshape(shape)
