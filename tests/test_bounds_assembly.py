"""Bounds of the warp-sliced row assembly (k_assemble_rows) and the BCRS3 fill
(k_fill_bcrs3), checked on the host by enumerating the kernels' index
arithmetic for many shapes.

Row assembly: one warp per 32 consecutive rows; each row's start is the
closed-form prefix of the per-axis neighbour counts (2 at an end of an axis,
3 inside), each lane writes its row into the warp's shared slice of 32 x 27
entries at the exclusive scan of the row lengths, and the warp stores the
slice at the first row's start.  Checked: the closed-form starts equal the
oracle's count-and-scan row pointer (Fig 3.6) bit for bit, every slice fits
the 864-entry shared buffer, consecutive warps' stores tile [0, nnz) without
gap or overlap, and nnz fits the int32 row pointer up to N = 429.

BCRS3 fill: per row, segments start at the first unconsumed column c, moved
left to n_cols - 3 at the last columns, and take every column <= c + 2; the
three-entry segment buffer is indexed by column - start.  Checked: that index
is 0, 1 or 2 for every entry, every start is a legal segment start, and a
row needs at most nine segments (the slice widths the conversion plans for)."""
import numpy as np
import pytest

import oracle

ASM_SLICE = 32 * 27


def axis_count(i, n):
    return np.where((i == 0) | (i == n), 2, 3).astype(np.int64)


def axis_prefix(i):
    return np.where(i == 0, 0, 3 * i.astype(np.int64) - 1)


def closed_form_starts(nx, ny, nz):
    nxn, nyn = nx + 1, ny + 1
    i = np.arange(nxn * nyn * (nz + 1), dtype=np.int64)
    ix, iy, iz = i % nxn, (i // nxn) % nyn, i // (nxn * nyn)
    cx, cy = 3 * nx + 1, 3 * ny + 1
    start = (cx * cy * axis_prefix(iz) + cx * axis_count(iz, nz) * axis_prefix(iy)
             + axis_count(iy, ny) * axis_count(iz, nz) * axis_prefix(ix))
    cnt = axis_count(ix, nx) * axis_count(iy, ny) * axis_count(iz, nz)
    return start, cnt


SHAPES = [(1, 1, 1), (2, 1, 1), (1, 1, 3), (4, 4, 4), (5, 3, 2), (31, 1, 2), (33, 17, 9), (30, 30, 30),
          (16, 64, 3)]


@pytest.mark.parametrize("dims", SHAPES)
def test_row_assembly_starts_slices_and_stores(dims):
    start, cnt = closed_form_starts(*dims)
    rp, cols = oracle.pattern(*dims)
    m, nnz = start.size, rp[-1]
    assert np.array_equal(start, rp[:-1]) and start[-1] + cnt[-1] == nnz
    # per warp: the slice of 32 rows fits the shared buffer; stores tile [0, nnz)
    pad = (-m) % 32
    c = np.concatenate([cnt, np.zeros(pad, dtype=np.int64)]).reshape(-1, 32)
    total = c.sum(axis=1)
    assert total.max() <= ASM_SLICE
    s0 = start[::32]
    assert s0[0] == 0 and np.array_equal(s0[1:], s0[:-1] + total[:-1])
    assert s0[-1] + total[-1] == nnz
    # each lane's place in its slice: exclusive scan, in [0, total)
    off = np.cumsum(c, axis=1) - c
    assert np.all(off + c <= total[:, None])


def test_row_pointer_fits_int32_up_to_n429():
    for n in (256, 400, 429, 430):
        nnz = (3 * n + 1) ** 3
        assert (nnz < 2 ** 31) == (n <= 429)
    start, cnt = closed_form_starts(429, 429, 2)
    assert start.max() + cnt.max() < 2 ** 31


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (4, 3, 5), (9, 1, 4), (17, 9, 23), (30, 30, 30)])
def test_bcrs3_segment_indices(dims):
    rp, cols = oracle.pattern(*dims)
    n_cols = rp.size - 1
    cmax = n_cols - 3
    widths = []
    for r in range(n_cols):
        j, hi, nseg = rp[r], rp[r + 1], 0
        while j < hi:
            c = cols[j]
            start = min(c, cmax)
            assert 0 <= start <= cmax
            while j < hi and cols[j] <= c + 2:
                assert 0 <= cols[j] - start <= 2
                j += 1
            nseg += 1
        widths.append(nseg)
    assert max(widths) <= 9
