"""Seeded synthetic inputs shared by the GPU tests, the oracle tests and the
benchmark.  Nothing here computes any part of the method: it only draws the
inputs (random vectors, random Dirichlet face data, mesh sizes for batches).

Face data recipe (random Dirichlet boundary values for the batched and
warm-start forms): every face of the cube gets i.i.d. U[0,1] draws, one per
face node, then three passes of a 3x3 mean whose window is clipped to the face
(each output is the mean of the in-face neighbours).  The generator is numpy's
PCG64 seeded with (base_seed, system index).  Faces are concatenated in the
order x0, x1, y0, y1, z0, z1; an x face is indexed iy + (ny+1) iz, a y face
ix + (nx+1) iz and a z face ix + (nx+1) iy.
"""
from __future__ import annotations

import numpy as np


def rng(*seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(list(seed)))


def random_vector(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n i.i.d. U[lo, hi) FP64 values."""
    return rng(seed, n).uniform(lo, hi, size=n)


def _box_mean_clipped(a: np.ndarray) -> np.ndarray:
    """One pass of a 3x3 mean, window clipped to the array (divide by in-array count)."""
    s = np.zeros_like(a)
    c = np.zeros_like(a)
    ny, nx = a.shape
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ys0, ys1 = max(0, dy), ny + min(0, dy)
            xs0, xs1 = max(0, dx), nx + min(0, dx)
            yd0, yd1 = max(0, -dy), ny + min(0, -dy)
            xd0, xd1 = max(0, -dx), nx + min(0, -dx)
            s[yd0:yd1, xd0:xd1] += a[ys0:ys1, xs0:xs1]
            c[yd0:yd1, xd0:xd1] += 1.0
    return s / c


def face_data(base_seed: int, index: int, nx: int, ny: int, nz: int,
              passes: int = 3) -> np.ndarray:
    """Concatenated random Dirichlet values for the six faces of an nx x ny x nz mesh."""
    g = rng(base_seed, index)
    shapes = [(nz + 1, ny + 1)] * 2 + [(nz + 1, nx + 1)] * 2 + [(ny + 1, nx + 1)] * 2
    out = []
    for shp in shapes:
        f = g.uniform(0.0, 1.0, size=shp)
        for _ in range(passes):
            f = _box_mean_clipped(f)
        out.append(f.ravel())
    return np.concatenate(out)


def minife_face_data(nx: int, ny: int, nz: int) -> np.ndarray:
    """Face array of the paper's boundary data: 1 on the x = 1 face, 0 on the others.

    Applied in face order, the y and z faces (0) overwrite the x = 1 face on the
    shared edges; the default problem (no face array) instead keeps the whole
    closed plane x = 1 at 1.
    """
    nyz, nxz, nxy = (ny + 1) * (nz + 1), (nx + 1) * (nz + 1), (nx + 1) * (ny + 1)
    out = np.zeros(2 * (nyz + nxz + nxy))
    out[nyz:2 * nyz] = 1.0
    return out


def batched_sizes(seed: int = 0, count: int = 64, lo: int = 32, hi: int = 128) -> np.ndarray:
    """Mesh sizes N ~ U{lo..hi} (inclusive) for a batch of cubic meshes."""
    return rng(seed).integers(lo, hi + 1, size=count)
