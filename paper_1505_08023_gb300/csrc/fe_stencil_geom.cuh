// fe_stencil_geom.cuh -- tile geometry and index arithmetic of the matrix-free
// operator (fe_stencil.cu): the interior tile columns, the staged halo tile and
// its slots, the boundary-row enumeration and the blocks' work ranges.  Plain
// C++ apart from the host/device qualifiers, so that a host program can walk
// the kernels' index arithmetic for bounds and coverage checks.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define FE_HD __host__ __device__
#else
#define FE_HD
#endif

namespace fe {

constexpr int kStWarps = 8;              // warps per block (the CG kernels' block)
constexpr int kStThreads = 32 * kStWarps;
constexpr int kStX = 32;                 // tile width along x: one warp
constexpr int kStR = 2;                  // rows per warp
constexpr int kStY = kStWarps * kStR;    // tile height along y
constexpr int kStPitch = kStX + 2;       // staged row with its halo
constexpr int kStElems = kStPitch * (kStY + 2);
constexpr int kStBuf = 2 * kStElems + (kStY + 2) * kStX;   // two staged planes + their row sums

struct StencilGeom {
    int nx, ny, nz;          // elements per axis
    int ntx, nty;            // interior tile columns along x and y
    long long cols;          // ntx * nty
    long long work;          // cols * (nz - 1): (column, interior plane) pairs
    long long n_bc;          // boundary rows
    long long m;             // rows
    double c[8];             // coefficient classes, k = |dx| + 2|dy| + 4|dz|
};

// Boundary row number q in [0, n_bc) -> node id.  Lines along x first: the
// lines with iz in {0, nz} or iy in {0, ny} are boundary from end to end
// (2 (ny+1) + 2 (nz-1) lines of nx+1 nodes); every other line contributes
// its two end nodes ix = 0 and ix = nx.
FE_HD inline long long bc_node(int nx, int ny, int nz, long long q) {
    const long long nxn = nx + 1, nyn = ny + 1, nzn = nz + 1;
    const long long full = 2 * nyn + 2 * (nzn > 2 ? nzn - 2 : 0);
    long long ix, iy, iz;
    if (q < full * nxn) {
        const long long l = q / nxn;
        ix = q - l * nxn;
        if (l < 2 * nyn) {
            iz = l < nyn ? 0 : nz;
            iy = l < nyn ? l : l - nyn;
        } else {
            const long long l2 = l - 2 * nyn;
            iz = 1 + l2 / 2;
            iy = (l2 & 1) ? ny : 0;
        }
    } else {
        const long long q2 = q - full * nxn, l = q2 / 2;
        ix = (q2 & 1) ? nx : 0;
        iy = 1 + l % (nyn - 2);
        iz = 1 + l / (nyn - 2);
    }
    return ix + nxn * (iy + nyn * iz);
}

FE_HD inline long long bc_count(int nx, int ny, int nz) {
    const long long nxn = nx + 1, nyn = ny + 1, nzn = nz + 1;
    const long long full = 2 * nyn + 2 * (nzn > 2 ? nzn - 2 : 0);
    const long long inner = (nyn > 2 && nzn > 2) ? (nyn - 2) * (nzn - 2) : 0;
    return full * nxn + 2 * inner;
}

// Staging slot: element e of the (kStY + 2) x kStPitch halo tile of the column
// whose first owned node is (x0, y0); `ok` is false for boundary nodes (x or
// y on a face) and nodes past the mesh, which are staged as 0.
struct StageSlot {
    int off;   // node offset within a plane ((nx+1)(ny+1) <= INT32_MAX, checked on the host)
    bool ok;
};

FE_HD inline StageSlot stage_slot(int nx, int ny, int x0, int y0, int e) {
    StageSlot s;
    const int ey = e / kStPitch, ex = e - ey * kStPitch;
    const int gx = x0 - 1 + ex, gy = y0 - 1 + ey;
    s.ok = e < kStElems && gx >= 1 && gx < nx && gy >= 1 && gy < ny;
    s.off = s.ok ? gx + (nx + 1) * gy : 0;
    return s;
}

// Staging: every thread stages its own kStR nodes (the tile's elements
// (kStR warp + r + 1, lane + 1)), and threads 0 .. kStHalo-1 one halo node
// each: the rows above and below the tile, then the two ends of each owned row.
constexpr int kStHalo = 2 * kStPitch + 2 * kStY;
static_assert(kStHalo <= kStThreads, "one halo node per thread at most");

FE_HD inline int halo_elem(int h) {
    if (h < kStPitch) return h;
    if (h < 2 * kStPitch) return (kStY + 1) * kStPitch + (h - kStPitch);
    const int k = h - 2 * kStPitch;
    return (1 + (k >> 1)) * kStPitch + ((k & 1) ? kStPitch - 1 : 0);
}

// The block's share of the (column, plane) work: one contiguous range of the
// column-major order, so a block marches at most a few column segments.
FE_HD inline void block_range(const StencilGeom &g, int block, int nblocks, long long *lo,
                                            long long *hi) {
    *lo = g.work * block / nblocks;
    *hi = g.work * (block + 1) / nblocks;
}

// Geometry of the nx x ny x nz box mesh and the operator's coefficient
// classes; false for sizes the kernels do not take.
inline bool stencil_geom(int nx, int ny, int nz, StencilGeom *g) {
    if (nx < 1 || ny < 1 || nz < 1) return false;
    if ((long long)(nx + 1) * (ny + 1) > INT32_MAX) return false;   // plane offsets are int32
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->ntx = (nx - 1 + kStX - 1) / kStX;
    g->nty = (ny - 1 + kStY - 1) / kStY;
    g->cols = (long long)g->ntx * g->nty;
    g->work = g->cols * (nz - 1);
    g->m = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    g->n_bc = bc_count(nx, ny, nz);
    const double h[3] = {1.0 / nx, 1.0 / ny, 1.0 / nz};
    double M[3][2], L[3][2];  // [axis][|offset|]
    for (int a = 0; a < 3; ++a) {
        M[a][0] = 2.0 * h[a] / 3.0;
        M[a][1] = h[a] / 6.0;
        L[a][0] = 2.0 / h[a];
        L[a][1] = -1.0 / h[a];
    }
    for (int k = 0; k < 8; ++k) {
        const int bx = k & 1, by = (k >> 1) & 1, bz = k >> 2;
        g->c[k] = L[0][bx] * M[1][by] * M[2][bz] + M[0][bx] * L[1][by] * M[2][bz] + M[0][bx] * M[1][by] * L[2][bz];
    }
    return true;
}

}  // namespace fe
