// Host walk of the matrix-free kernels' index arithmetic (fe_stencil.cu):
// for every block of a grid and every thread of the block it replays the
// loop skeleton of the operator pass (stencil_pass -> stencil_column, then
// stencil_bc_rows) with the kernels' own index functions from
// fe_stencil_geom.cuh, and checks
//   * every global load and store index lies in [0, m);
//   * every shared-memory index lies in the staged tiles / row-sum buffer;
//   * every interior node is written by exactly one (block, thread, plane) and
//     every boundary node by exactly one boundary-row visit, so the pass
//     covers the m rows once;
//   * the halo slots a thread stages are the tile elements the sums read.
// Usage: stencil_index_check nx ny nz nblocks [nblocks ...]; prints one line
// per grid and exits 1 on the first violation.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "fe_stencil_geom.cuh"

using namespace fe;

static long long g_checks = 0;

#define CHECK(cond, ...)                                     \
    do {                                                     \
        ++g_checks;                                          \
        if (!(cond)) {                                       \
            std::fprintf(stderr, "violation: " __VA_ARGS__); \
            std::fprintf(stderr, "\n");                      \
            std::exit(1);                                    \
        }                                                    \
    } while (0)

static bool interior(const StencilGeom &g, long long i) {
    const long long nxn = g.nx + 1, nyn = g.ny + 1;
    const long long ix = i % nxn, iy = (i / nxn) % nyn, iz = i / (nxn * nyn);
    return ix > 0 && ix < g.nx && iy > 0 && iy < g.ny && iz > 0 && iz < g.nz;
}

// shared-memory index of a staged tile element in buffer `par`
static void shared_tile(int par, int e, const char *what) {
    CHECK(e >= 0 && e < kStElems, "%s: tile element %d outside [0, %d)", what, e, kStElems);
    const int idx = par * kStElems + e;
    CHECK(idx >= 0 && idx < 2 * kStElems, "%s: shared index %d", what, idx);
}

static void shared_rowsum(int r, int lane, const char *what) {
    const int idx = 2 * kStElems + r * kStX + lane;
    CHECK(r >= 0 && r < kStY + 2 && idx < kStBuf, "%s: row-sum index %d (row %d)", what, idx, r);
}

static void global(const StencilGeom &g, long long i, const char *what) {
    CHECK(i >= 0 && i < g.m, "%s: global index %lld outside [0, %lld)", what, i, g.m);
}

// One column t, planes zlo .. zhi - 1 (interior planes), every thread of the
// block; `written` counts the writes of each row.
static void column(const StencilGeom &g, long long t, int zlo, int zhi, std::vector<unsigned char> &written) {
    const int tx = (int)(t % g.ntx), ty = (int)(t / g.ntx);
    const int x0 = 1 + kStX * tx, y0 = 1 + kStY * ty;
    const long long sxy = (long long)(g.nx + 1) * (g.ny + 1);
    for (int tid = 0; tid < kStThreads; ++tid) {
        const int lane = tid & 31, warp = tid >> 5;
        const int sr0 = kStR * warp + 1;
        const int c0 = sr0 * kStPitch + lane + 1, c1 = c0 + kStPitch;
        const bool has_h = tid < kStHalo;
        const int eh = has_h ? halo_elem(tid) : 0;
        const StageSlot s0 = stage_slot(g.nx, g.ny, x0, y0, c0);
        const StageSlot s1 = stage_slot(g.nx, g.ny, x0, y0, c1);
        const StageSlot sh = has_h ? stage_slot(g.nx, g.ny, x0, y0, eh) : StageSlot{0, false};
        if (has_h) {
            // a halo element is on the tile's border: the rows above and below,
            // or the first / last column of an owned row
            const int ey = eh / kStPitch, ex = eh % kStPitch;
            CHECK(ey == 0 || ey == kStY + 1 || ex == 0 || ex == kStPitch - 1, "halo element %d inside the tile", eh);
        }
        auto fetch = [&](int q) {
            const bool zin = q >= 1 && q < g.nz;
            const long long b = sxy * q;
            if (zin && s0.ok) global(g, b + s0.off, "fetch s0");
            if (zin && s1.ok) global(g, b + s1.off, "fetch s1");
            if (zin && sh.ok) global(g, b + sh.off, "fetch halo");
        };
        fetch(zlo - 1);
        int par = 0;
        for (int q = zlo - 1; q <= zhi; ++q) {
            shared_tile(par, c0, "stage c0");
            shared_tile(par, c1, "stage c1");
            if (has_h) shared_tile(par, eh, "stage halo");
            if (q >= zlo && q < zhi) {                       // x with the plane loads (CG pass)
                if (s0.ok) global(g, sxy * q + s0.off, "x s0");
                if (s1.ok) global(g, sxy * q + s1.off, "x s1");
            }
            if (q < zhi) fetch(q + 1);
            shared_tile(par, c0 - 1, "Sx c0-1");
            shared_tile(par, c0 + 1, "Sx c0+1");
            shared_tile(par, c1 - 1, "Sx c1-1");
            shared_tile(par, c1 + 1, "Sx c1+1");
            shared_rowsum(sr0, lane, "Sx store 0");
            shared_rowsum(sr0 + 1, lane, "Sx store 1");
            if (warp < 2) {
                const int r = warp == 0 ? 0 : kStY + 1;
                shared_rowsum(r, lane, "halo Sx store");
                shared_tile(par, r * kStPitch + lane, "halo Sx left");
                shared_tile(par, r * kStPitch + lane + 2, "halo Sx right");
            }
            shared_rowsum(sr0 - 1, lane, "D above");
            shared_rowsum(sr0 + 2, lane, "D below");
            shared_tile(par, c0 - kStPitch, "Sy above");
            shared_tile(par, c1 + kStPitch, "Sy below");
            if (q > zlo) {
                for (const StageSlot *so : {&s0, &s1}) {
                    if (!so->ok) continue;
                    const long long i = sxy * (q - 1) + so->off;
                    global(g, i, "row out");
                    CHECK(interior(g, i), "row out %lld is not an interior node", i);
                    CHECK(written[i] == 0, "row %lld written twice", i);
                    written[i] = 1;
                }
            }
            par ^= 1;
        }
    }
}

static void pass(const StencilGeom &g, int nblocks, std::vector<unsigned char> &written) {
    const int nzi = g.nz - 1;
    for (int b = 0; b < nblocks; ++b) {
        long long lo, hi;
        block_range(g, b, nblocks, &lo, &hi);
        CHECK(lo <= hi && hi <= g.work, "block %d range [%lld, %lld)", b, lo, hi);
        while (lo < hi) {
            const long long t = lo / nzi;
            const int z0 = (int)(lo - t * nzi);
            const long long left = hi - lo;
            const int z1 = (int)((nzi - z0) < left ? nzi : z0 + left);
            CHECK(t < g.cols && z0 < z1 && z1 <= nzi, "segment t %lld z [%d, %d)", t, z0, z1);
            column(g, t, 1 + z0, 1 + z1, written);
            lo += z1 - z0;
        }
    }
    // boundary rows, grid-strided over all threads
    for (long long q = 0; q < g.n_bc; ++q) {
        const long long i = bc_node(g.nx, g.ny, g.nz, q);
        global(g, i, "boundary row");
        CHECK(!interior(g, i), "boundary row %lld is interior", i);
        CHECK(written[i] == 0, "boundary row %lld written twice", i);
        written[i] = 1;
    }
}

int main(int argc, char **argv) {
    if (argc < 5) {
        std::fprintf(stderr, "usage: %s nx ny nz nblocks [nblocks ...]\n", argv[0]);
        return 2;
    }
    const int nx = std::atoi(argv[1]), ny = std::atoi(argv[2]), nz = std::atoi(argv[3]);
    StencilGeom g;
    if (!stencil_geom(nx, ny, nz, &g)) {
        std::fprintf(stderr, "geometry rejected\n");
        return 2;
    }
    const long long inner = (long long)(nx > 1 ? nx - 1 : 0) * (ny > 1 ? ny - 1 : 0) * (nz > 1 ? nz - 1 : 0);
    CHECK(g.n_bc + inner == g.m, "boundary count %lld + interior %lld != m %lld", g.n_bc, inner, g.m);
    for (int a = 4; a < argc; ++a) {
        const int nb = std::atoi(argv[a]);
        std::vector<unsigned char> written((size_t)g.m, 0);
        pass(g, nb, written);
        for (long long i = 0; i < g.m; ++i) CHECK(written[i] == 1, "row %lld not written", i);
        std::printf("ok %d %d %d blocks %d: %lld checks\n", nx, ny, nz, nb, g_checks);
    }
    return 0;
}
