// fe_cg_batched.cu -- many independent CG solves (meshes of different sizes,
// different boundary data) in one persistent cooperative launch.
//
// Systems with the same matrix form a group; a group's systems are cut into
// chunks of up to KRHS right-hand sides, and a chunk's SpMV is an SpMM: each
// matrix slot is loaded once and applied to every active right-hand side of
// the chunk.  The work of a phase is the list of units (chunk, slice) of the
// chunks that still hold an unconverged system, in chunk order; block b takes
// units [b U / G, (b+1) U / G) of the U active units.  Every block derives
// that list from the same per-system flags, so the partition is identical in
// all blocks and shrinks as systems converge.  Block ranges are contiguous,
// so the blocks that touch one system form a contiguous range, and a system's
// dot product is the sum of their partials in block order; inside a block the
// warps' partials are summed in warp order.  No atomics: reruns give the same
// bits.  All systems step in lockstep; each has its own alpha, beta, stopping
// test and status, as fe_cg_solve would give it.
//
// Two step forms (template SR): textbook CG (passes SpMV w = A p with p.w,
// x/r update with r.r, p update: three barriers per step) and the
// single-reduction form of fe_cg_solve_sr (SpMV w = A r with r.r and w.r, then
// one streaming pass p = r + beta p, s = w + beta s, x += alpha p,
// r -= alpha s: two barriers per step).
#include <vector>
#include <algorithm>

#include "fe_cg_common.cuh"

namespace fe {

constexpr int kBatchMaxSystems = 256;
constexpr int kBatchMaxTouch = 32;   // systems one block may touch in one phase
constexpr int kBatchThreads = kCgThreads;

struct BatchSysDev {
    const double *b;
    double *x, *r, *p, *w, *s;   // s = A p (single-reduction form only)
    int chunk;
    int pad;
};

struct BatchChunkDev {
    fe_matrix A;
    int first_sys;
    int n_rhs;
    int n_slices;
    int pad;
};

struct BatchArgs {
    const BatchSysDev *sys;
    const BatchChunkDev *chunks;
    int n_sys, n_chunks;
    double *part;          // [2 rounds][2 values][G][kBatchMaxTouch]
    int *first_sys_of;     // [2 rounds][G]
    CgCtrl *ctrl;
    int *out_status, *out_iters;
    double *out_rr, *out_bb;
    double tol2;
    int maxit;
    int max_blocks;
    long long timeout_ns;
};

struct BatchShared {
    CgBlockState st;
    long long unit_start[kBatchMaxSystems + 1];
    long long n_units;
    int n_active;
    int touch_overflow;
    int active[kBatchMaxSystems];
    int mask[kBatchMaxSystems];        // systems the current pass works on
    int status[kBatchMaxSystems];
    int iters[kBatchMaxSystems];
    double rr[kBatchMaxSystems], bb[kBatchMaxSystems];
    double coef[kBatchMaxSystems];     // alpha or beta of the current pass
    double coef2[kBatchMaxSystems];    // beta of the single-reduction update
    double red[2][kBatchMaxSystems];   // reduced dot products of the last pass
    double wpart[2][kCgWarps][kBatchMaxTouch];
};

__device__ __forceinline__ long long block_start(long long U, int b, int G) { return (U * b) / G; }
__device__ __forceinline__ int block_of_unit(long long U, long long u, int G) {
    return (int)(((u + 1) * G - 1) / U);
}

// Unit list of the chunks holding a system marked in sh.mask (warp 0 runs a
// prefix sum over the chunks, 32 at a time).
__device__ __forceinline__ void batch_plan(const BatchArgs &a, BatchShared &sh) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        long long base = 0;
        for (int c0 = 0; c0 < a.n_chunks; c0 += 32) {
            const int c = c0 + lane;
            long long len = 0;
            if (c < a.n_chunks) {
                const int f = a.chunks[c].first_sys, nr = a.chunks[c].n_rhs;
                bool any = false;
                for (int j = 0; j < nr; ++j) any |= sh.mask[f + j] != 0;
                if (any) len = a.chunks[c].n_slices;
            }
            long long incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (c < a.n_chunks) sh.unit_start[c] = base + incl - len;
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            sh.unit_start[a.n_chunks] = base;
            sh.n_units = base;
        }
    }
    __syncthreads();
}

// Chunk holding unit u: the last chunk whose range starts at or before u and is non-empty.
__device__ __forceinline__ int chunk_of_unit(const BatchShared &sh, int n_chunks, long long u) {
    int lo = 0, hi = n_chunks - 1;
    while (lo < hi) {  // largest c with unit_start[c] <= u
        const int mid = (lo + hi + 1) >> 1;
        if (sh.unit_start[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;  // empty chunks share their start with the next one, so the largest is non-empty
}

// SpMM of one slice for up to KRHS right-hand sides (BCRS3 or SELL, FP64 values).
template <int FMT, int KRHS>
__device__ __forceinline__ void slice_spmm(const fe_matrix &A, int s, int lane, const double *const *xs,
                                           const bool *on, double *acc) {
#pragma unroll
    for (int j = 0; j < KRHS; ++j) acc[j] = 0.0;
    const int64_t b = A.d_slice_ptr[s];
    const int w = (int)((A.d_slice_ptr[s + 1] - b) >> 5);
    const int32_t *c = A.d_cols + b + lane;
    if constexpr (FMT == FE_FMT_BCRS3) {
        const double *v = reinterpret_cast<const double *>(A.d_vals) + 3 * b + lane;
        int k = 0;
        constexpr int U = 3;
        for (; k + U <= w; k += U) {
            int32_t col[U];
            double vv[U][3];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                col[u] = ld_stream(c + 32 * (k + u));
#pragma unroll
                for (int t = 0; t < 3; ++t) vv[u][t] = ld_stream(v + 96 * (k + u) + 32 * t);
            }
#pragma unroll
            for (int j = 0; j < KRHS; ++j) {
                if (!on[j]) continue;
                double xx[U][3];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int t = 0; t < 3; ++t) xx[u][t] = xs[j][col[u] + t];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int t = 0; t < 3; ++t) acc[j] = fma(vv[u][t], xx[u][t], acc[j]);
            }
        }
        for (; k < w; ++k) {
            const int32_t col = ld_stream(c + 32 * k);
            const double v0 = ld_stream(v + 96 * k), v1 = ld_stream(v + 96 * k + 32),
                         v2 = ld_stream(v + 96 * k + 64);
#pragma unroll
            for (int j = 0; j < KRHS; ++j) {
                if (!on[j]) continue;
                const double *x = xs[j] + col;
                acc[j] = fma(v0, x[0], acc[j]);
                acc[j] = fma(v1, x[1], acc[j]);
                acc[j] = fma(v2, x[2], acc[j]);
            }
        }
    } else {
        const double *v = reinterpret_cast<const double *>(A.d_vals) + b + lane;
        int k = 0;
        constexpr int U = 9;
        for (; k + U <= w; k += U) {
            int32_t col[U];
            double vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                col[u] = ld_stream(c + 32 * (k + u));
                vv[u] = ld_stream(v + 32 * (k + u));
            }
#pragma unroll
            for (int j = 0; j < KRHS; ++j) {
                if (!on[j]) continue;
                double xx[U];
#pragma unroll
                for (int u = 0; u < U; ++u) xx[u] = xs[j][col[u]];
#pragma unroll
                for (int u = 0; u < U; ++u) acc[j] = fma(vv[u], xx[u], acc[j]);
            }
        }
        for (; k < w; ++k) {
            const int32_t col = ld_stream(c + 32 * k);
            const double vv = ld_stream(v + 32 * k);
#pragma unroll
            for (int j = 0; j < KRHS; ++j)
                if (on[j]) acc[j] = fma(vv, xs[j][col], acc[j]);
        }
    }
}

enum BatchPass { kInit = 0, kSpmv = 1, kUpdateXR = 2, kUpdateP = 3, kZeroX = 4, kSpmvR = 5,
                 kUpdateSR = 6 };

// One pass over the block's units for the systems in sh.mask.  Passes with a
// dot product leave the per-system block partials in global memory
// (part[round][v][block][t]); returns false if a barrier gave up.
template <int FMT, int KRHS, bool SR>
__device__ bool batch_pass(const BatchArgs &a, BatchShared &sh, int pass) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    batch_plan(a, sh);
    const long long U = sh.n_units;
    const bool has_dots = pass == kInit || pass == kSpmv || pass == kUpdateXR || pass == kSpmvR;
    for (int i = threadIdx.x; i < 2 * kCgWarps * kBatchMaxTouch; i += blockDim.x)
        (&sh.wpart[0][0][0])[i] = 0.0;
    __syncthreads();
    const long long u_begin = U > 0 ? block_start(U, blockIdx.x, G) : 0;
    const long long u_end = U > 0 ? block_start(U, blockIdx.x + 1, G) : 0;
    const int first_sys = (u_begin < u_end) ? a.chunks[chunk_of_unit(sh, a.n_chunks, u_begin)].first_sys : 0;
    if (pass == kInit || pass == kSpmv || pass == kSpmvR) {
        // warp per slice; the chunk lookup is reused while the warp stays in one
        // chunk, and the dot-product partials stay in the lanes' registers until
        // the warp leaves the chunk (then one butterfly per system and partial)
        const bool two = pass != kSpmv;     // passes with a second dot product
        int c = -1;
        long long c_lo = 0, c_hi = 0;
        double pd0[KRHS], pd1[KRHS];
#pragma unroll
        for (int j = 0; j < KRHS; ++j) pd0[j] = pd1[j] = 0.0;
        // adds the warp's partials of chunk c to shared memory (fixed order)
        auto flush = [&](int cc) {
            if (cc < 0) return;
            const BatchChunkDev &fc = a.chunks[cc];
#pragma unroll
            for (int j = 0; j < KRHS; ++j) {
                if (j >= fc.n_rhs || !sh.mask[fc.first_sys + j]) continue;
                const double d0 = warp_sum(pd0[j]);
                const double d1 = two ? warp_sum(pd1[j]) : 0.0;
                const int t = fc.first_sys + j - first_sys;
                if (lane == 0) {
                    if (t >= 0 && t < kBatchMaxTouch) {
                        sh.wpart[0][warp][t] += d0;
                        sh.wpart[1][warp][t] += d1;
                    } else {
                        sh.touch_overflow = 1;
                    }
                }
                pd0[j] = pd1[j] = 0.0;
            }
        };
        for (long long u = u_begin + warp; u < u_end; u += kCgWarps) {
            if (u < c_lo || u >= c_hi) {
                flush(c);
                c = chunk_of_unit(sh, a.n_chunks, u);
                c_lo = sh.unit_start[c];
                c_hi = c_lo + a.chunks[c].n_slices;
            }
            const BatchChunkDev &ch = a.chunks[c];
            const int slice = (int)(u - c_lo);
            const int row = slice * kSlice + lane;
            const bool in = row < (int)ch.A.n_rows;
            bool on[KRHS];
            const double *xin[KRHS];
            double acc[KRHS];
#pragma unroll
            for (int j = 0; j < KRHS; ++j) {
                on[j] = j < ch.n_rhs && sh.mask[ch.first_sys + j] != 0;
                xin[j] = nullptr;
                if (on[j])
                    xin[j] = (pass == kInit) ? a.sys[ch.first_sys + j].x
                                             : (pass == kSpmvR ? a.sys[ch.first_sys + j].r
                                                               : a.sys[ch.first_sys + j].p);
            }
            slice_spmm<FMT, KRHS>(ch.A, slice, lane, xin, on, acc);
#pragma unroll
            for (int j = 0; j < KRHS; ++j) {
                if (!on[j] || !in) continue;
                const BatchSysDev &sd = a.sys[ch.first_sys + j];
                if (pass == kInit) {
                    const double bi = sd.b[row], ri = bi - acc[j];
                    sd.r[row] = ri;
                    if (SR) {
                        sd.p[row] = 0.0;
                        sd.s[row] = 0.0;
                    } else {
                        sd.p[row] = ri;
                    }
                    pd0[j] = fma(ri, ri, pd0[j]);
                    pd1[j] = fma(bi, bi, pd1[j]);
                } else if (pass == kSpmvR) {
                    const double ri = sd.r[row];
                    sd.w[row] = acc[j];
                    pd0[j] = fma(ri, ri, pd0[j]);
                    pd1[j] = fma(acc[j], ri, pd1[j]);
                } else {
                    sd.w[row] = acc[j];
                    pd0[j] = fma(sd.p[row], acc[j], pd0[j]);
                }
            }
        }
        flush(c);
    } else {
        // streaming passes: the block's unit range is a contiguous row range of
        // each chunk it touches; all threads stream each system's rows there in
        // 16-byte packs (row ranges start on 32-row boundaries)
        long long u = u_begin;
        while (u < u_end) {
            const int c = chunk_of_unit(sh, a.n_chunks, u);
            const BatchChunkDev &ch = a.chunks[c];
            const long long c_lo = sh.unit_start[c];
            const long long u_stop = (c_lo + ch.n_slices < u_end) ? c_lo + ch.n_slices : u_end;
            const int row0 = (int)(u - c_lo) * kSlice;
            int row1 = (int)(u_stop - c_lo) * kSlice;
            if (row1 > (int)ch.A.n_rows) row1 = (int)ch.A.n_rows;
            for (int j = 0; j < ch.n_rhs; ++j) {
                const int s = ch.first_sys + j;
                if (!sh.mask[s]) continue;
                const BatchSysDev &sd = a.sys[s];
                const int npk = (row1 - row0) >> 1;
                double d0 = 0.0;
                if (pass == kUpdateXR) {
                    const double al = sh.coef[s];
                    double2 *x2 = reinterpret_cast<double2 *>(sd.x + row0);
                    double2 *r2 = reinterpret_cast<double2 *>(sd.r + row0);
                    const double2 *p2 = reinterpret_cast<const double2 *>(sd.p + row0);
                    const double2 *w2 = reinterpret_cast<const double2 *>(sd.w + row0);
                    for (int q = threadIdx.x; q < npk; q += blockDim.x) {
                        double2 xv = x2[q], rv = r2[q];
                        const double2 pv = p2[q], wv = w2[q];
                        xv.x = fma(al, pv.x, xv.x);
                        xv.y = fma(al, pv.y, xv.y);
                        rv.x = fma(-al, wv.x, rv.x);
                        rv.y = fma(-al, wv.y, rv.y);
                        x2[q] = xv;
                        r2[q] = rv;
                        d0 = fma(rv.x, rv.x, d0);
                        d0 = fma(rv.y, rv.y, d0);
                    }
                    for (int row = row0 + 2 * npk + threadIdx.x; row < row1; row += blockDim.x) {
                        sd.x[row] = fma(al, sd.p[row], sd.x[row]);
                        const double ri = fma(-al, sd.w[row], sd.r[row]);
                        sd.r[row] = ri;
                        d0 = fma(ri, ri, d0);
                    }
                } else if (pass == kUpdateSR) {
                    const double al = sh.coef[s], be = sh.coef2[s];
                    double2 *x2 = reinterpret_cast<double2 *>(sd.x + row0);
                    double2 *r2 = reinterpret_cast<double2 *>(sd.r + row0);
                    double2 *p2 = reinterpret_cast<double2 *>(sd.p + row0);
                    double2 *s2 = reinterpret_cast<double2 *>(sd.s + row0);
                    const double2 *w2 = reinterpret_cast<const double2 *>(sd.w + row0);
                    for (int q = threadIdx.x; q < npk; q += blockDim.x) {
                        double2 xv = x2[q], rv = r2[q], pv = p2[q], sv = s2[q];
                        const double2 wv = w2[q];
                        pv.x = fma(be, pv.x, rv.x);
                        pv.y = fma(be, pv.y, rv.y);
                        sv.x = fma(be, sv.x, wv.x);
                        sv.y = fma(be, sv.y, wv.y);
                        xv.x = fma(al, pv.x, xv.x);
                        xv.y = fma(al, pv.y, xv.y);
                        rv.x = fma(-al, sv.x, rv.x);
                        rv.y = fma(-al, sv.y, rv.y);
                        x2[q] = xv;
                        r2[q] = rv;
                        p2[q] = pv;
                        s2[q] = sv;
                    }
                    for (int row = row0 + 2 * npk + threadIdx.x; row < row1; row += blockDim.x) {
                        const double pi = fma(be, sd.p[row], sd.r[row]);
                        const double si = fma(be, sd.s[row], sd.w[row]);
                        sd.p[row] = pi;
                        sd.s[row] = si;
                        sd.x[row] = fma(al, pi, sd.x[row]);
                        sd.r[row] = fma(-al, si, sd.r[row]);
                    }
                } else if (pass == kUpdateP) {
                    const double be = sh.coef[s];
                    double2 *p2 = reinterpret_cast<double2 *>(sd.p + row0);
                    const double2 *r2 = reinterpret_cast<const double2 *>(sd.r + row0);
                    for (int q = threadIdx.x; q < npk; q += blockDim.x) {
                        double2 pv = p2[q];
                        const double2 rv = r2[q];
                        pv.x = fma(be, pv.x, rv.x);
                        pv.y = fma(be, pv.y, rv.y);
                        p2[q] = pv;
                    }
                    for (int row = row0 + 2 * npk + threadIdx.x; row < row1; row += blockDim.x)
                        sd.p[row] = fma(be, sd.p[row], sd.r[row]);
                } else {
                    for (int row = row0 + threadIdx.x; row < row1; row += blockDim.x) sd.x[row] = 0.0;
                }
                if (has_dots) {
                    d0 = warp_sum(d0);
                    const int t = s - first_sys;
                    if (lane == 0) {
                        if (t >= 0 && t < kBatchMaxTouch) sh.wpart[0][warp][t] += d0;
                        else sh.touch_overflow = 1;
                    }
                }
            }
            u = u_stop;
        }
    }
    if (!has_dots) return grid_barrier(a.ctrl, &sh.st, a.timeout_ns, -1);
    __syncthreads();
    const int rnd = sh.st.round & 1;
    double *part = a.part + (size_t)rnd * 2 * a.max_blocks * kBatchMaxTouch;
    if (threadIdx.x < kBatchMaxTouch) {
        double t0 = 0.0, t1 = 0.0;
#pragma unroll
        for (int w = 0; w < kCgWarps; ++w) {
            t0 += sh.wpart[0][w][threadIdx.x];
            t1 += sh.wpart[1][w][threadIdx.x];
        }
        __stcg(part + (size_t)blockIdx.x * kBatchMaxTouch + threadIdx.x, t0);
        __stcg(part + ((size_t)a.max_blocks + blockIdx.x) * kBatchMaxTouch + threadIdx.x, t1);
    }
    if (threadIdx.x == 0) __stcg(a.first_sys_of + rnd * a.max_blocks + blockIdx.x, first_sys);
    if (!grid_barrier(a.ctrl, &sh.st, a.timeout_ns, -1)) return false;
    // per system: sum the partials of the blocks that touched it, in block order
    const int *fsys = a.first_sys_of + rnd * a.max_blocks;
    for (int s = warp; s < a.n_sys; s += kCgWarps) {
        if (!sh.mask[s]) continue;
        const int c = a.sys[s].chunk;
        const long long u0 = sh.unit_start[c], u1 = u0 + a.chunks[c].n_slices - 1;
        const int b0 = block_of_unit(U, u0, G), b1 = block_of_unit(U, u1, G);
        double t0 = 0.0, t1 = 0.0;
        for (int bb = b0 + lane; bb <= b1; bb += 32) {
            const int t = s - __ldcg(fsys + bb);
            if (t >= 0 && t < kBatchMaxTouch) {
                t0 += __ldcg(part + (size_t)bb * kBatchMaxTouch + t);
                t1 += __ldcg(part + ((size_t)a.max_blocks + bb) * kBatchMaxTouch + t);
            }
        }
        t0 = warp_sum(t0);
        t1 = warp_sum(t1);
        if (lane == 0) {
            sh.red[0][s] = t0;
            sh.red[1][s] = t1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.st.round += 1;
    __syncthreads();
    return true;
}

template <int FMT, int KRHS, bool SR>
__global__ void __launch_bounds__(kBatchThreads, KRHS <= 2 ? 4 : 2) k_cg_batched(const BatchArgs a) {
    __shared__ BatchShared sh;
    const int n = a.n_sys;
    if (threadIdx.x == 0) {
        sh.st.target = 0;
        sh.st.round = 0;
        sh.st.k = 0;
        sh.st.ok = 1;
        sh.touch_overflow = 0;
    }
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        sh.active[s] = 1;
        sh.mask[s] = 1;
        sh.status[s] = FE_ERR_MAXIT;
        sh.iters[s] = 0;
    }
    bool alive = batch_pass<FMT, KRHS, SR>(a, sh, kInit);
    if (alive) {
        int any_zero = 0;
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            sh.rr[s] = sh.red[0][s];
            sh.bb[s] = sh.red[1][s];
            sh.mask[s] = 0;
            if (sh.bb[s] == 0.0) {          // b = 0: x = 0, no step
                sh.rr[s] = 0.0;
                sh.status[s] = FE_OK;
                sh.active[s] = 0;
                sh.mask[s] = 1;
                any_zero = 1;
            } else if (sh.rr[s] <= a.tol2 * sh.bb[s]) {
                sh.status[s] = FE_OK;
                sh.active[s] = 0;
            }
        }
        if (__syncthreads_or(any_zero)) alive = batch_pass<FMT, KRHS, SR>(a, sh, kZeroX);
    }
    bool first = true;
    while (alive && SR) {
        for (int s = threadIdx.x; s < n; s += blockDim.x) sh.mask[s] = sh.active[s];
        __syncthreads();
        int na = 0;
        for (int s = 0; s < n; ++s) na += sh.active[s];
        if (na == 0) break;
        // w = A r, gamma = r.r, delta = w.r
        if (!(alive = batch_pass<FMT, KRHS, SR>(a, sh, kSpmvR))) break;
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            if (!sh.active[s]) continue;
            const double gamma = sh.red[0][s], delta = sh.red[1][s];
            if (!first) sh.iters[s] += 1;
            double beta = 0.0, curv = delta;
            if (!first) {
                beta = gamma / sh.rr[s];
                curv = delta - beta * gamma / sh.coef[s];   // coef: alpha of the previous step
                if (!(curv > 0.0) || !(curv < INFINITY)) {  // lost its sign: restart the direction
                    beta = 0.0;
                    curv = delta;
                }
            }
            sh.rr[s] = gamma;
            if (gamma <= a.tol2 * sh.bb[s]) {
                sh.status[s] = FE_OK;
                sh.active[s] = 0;
            } else if (sh.iters[s] >= a.maxit) {
                sh.status[s] = FE_ERR_MAXIT;
                sh.active[s] = 0;
            } else if (!(curv > 0.0) || !(curv < INFINITY)) {
                sh.status[s] = FE_ERR_BREAKDOWN;
                sh.active[s] = 0;
            } else {
                sh.coef[s] = gamma / curv;
                sh.coef2[s] = beta;
            }
            sh.mask[s] = sh.active[s];
        }
        __syncthreads();
        na = 0;
        for (int s = 0; s < n; ++s) na += sh.active[s];
        if (na == 0) break;
        // p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s
        if (!(alive = batch_pass<FMT, KRHS, SR>(a, sh, kUpdateSR))) break;
        first = false;
    }
    while (alive && !SR) {
        for (int s = threadIdx.x; s < n; s += blockDim.x) sh.mask[s] = sh.active[s];
        __syncthreads();
        int na = 0;
        for (int s = 0; s < n; ++s) na += sh.active[s];
        if (na == 0) break;
        // w = A p, p.w
        if (!(alive = batch_pass<FMT, KRHS, SR>(a, sh, kSpmv))) break;
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            if (!sh.active[s]) continue;
            const double pw = sh.red[0][s];
            if (!(pw > 0.0) || !(pw < INFINITY)) {
                sh.status[s] = FE_ERR_BREAKDOWN;
                sh.active[s] = 0;
                sh.mask[s] = 0;
            } else {
                sh.coef[s] = sh.rr[s] / pw;
            }
        }
        // x += alpha p, r -= alpha w, r.r
        if (!(alive = batch_pass<FMT, KRHS, SR>(a, sh, kUpdateXR))) break;
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            if (!sh.active[s]) continue;
            const double rr_new = sh.red[0][s];
            sh.coef[s] = rr_new / sh.rr[s];
            sh.rr[s] = rr_new;
            sh.iters[s] += 1;
            if (rr_new <= a.tol2 * sh.bb[s]) {
                sh.status[s] = FE_OK;
                sh.active[s] = 0;
                sh.mask[s] = 0;
            } else if (sh.iters[s] >= a.maxit) {
                sh.status[s] = FE_ERR_MAXIT;
                sh.active[s] = 0;
                sh.mask[s] = 0;
            }
        }
        // p = r + beta p
        if (!(alive = batch_pass<FMT, KRHS, SR>(a, sh, kUpdateP))) break;
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            a.out_status[s] = !alive ? FE_ERR_TIMEOUT : (sh.touch_overflow ? FE_ERR_ARG : sh.status[s]);
            a.out_iters[s] = sh.iters[s];
            a.out_rr[s] = sh.rr[s];
            a.out_bb[s] = sh.bb[s];
        }
        if (threadIdx.x == 0) a.ctrl->status = alive ? FE_OK : FE_ERR_TIMEOUT;
    }
}

// ---------------------------------------------------------------- host side

// Workspace layout: control block, tables, partials, outputs, then r, p, w
// of every system.  Offsets depend only on n and max_blocks (and the matrix
// sizes for the vectors), so plan, launch and results agree.
struct Fixed {
    size_t sys, chunks, part, fsys, out_int, out_dbl, vecs;
};

static Fixed fixed_offsets(int n, int max_blocks) {
    Fixed F;
    size_t o = 256;
    F.sys = o;     o += align256(sizeof(BatchSysDev) * (size_t)n);
    F.chunks = o;  o += align256(sizeof(BatchChunkDev) * (size_t)n);
    F.part = o;    o += align256(sizeof(double) * 2 * 2 * (size_t)max_blocks * kBatchMaxTouch);
    F.fsys = o;    o += align256(sizeof(int) * 2 * (size_t)max_blocks);
    F.out_int = o; o += align256(sizeof(int) * 2 * (size_t)n);
    F.out_dbl = o; o += align256(sizeof(double) * 2 * (size_t)n);
    F.vecs = o;
    return F;
}

// Offsets of each system's r, p, w, s block (caller's numbering) and the total.
static size_t vector_offsets(int n, const fe_matrix *A, int max_blocks, std::vector<size_t> *off) {
    size_t o = fixed_offsets(n, max_blocks).vecs;
    for (int i = 0; i < n; ++i) {
        if (off) off->push_back(o);
        o += 4 * align256((size_t)A[i].n_slices * kSlice * sizeof(double));
    }
    return o;
}

// The kernel instance of (format, RHS chunk, method).
template <int FMT, int KRHS> static const void *kernel_of(int method) {
    return method == FE_BATCH_SINGLE_REDUCTION ? (const void *)k_cg_batched<FMT, KRHS, true>
                                               : (const void *)k_cg_batched<FMT, KRHS, false>;
}

static const void *batched_kernel(int fmt, int krhs, int method) {
    if (fmt == FE_FMT_BCRS3) {
        if (krhs == 1) return kernel_of<FE_FMT_BCRS3, 1>(method);
        if (krhs == 2) return kernel_of<FE_FMT_BCRS3, 2>(method);
        if (krhs == 4) return kernel_of<FE_FMT_BCRS3, 4>(method);
    } else if (fmt == FE_FMT_SELL) {
        if (krhs == 1) return kernel_of<FE_FMT_SELL, 1>(method);
        if (krhs == 2) return kernel_of<FE_FMT_SELL, 2>(method);
        if (krhs == 4) return kernel_of<FE_FMT_SELL, 4>(method);
    }
    return nullptr;
}

static BatchArgs args_of(const fe_batch_plan *plan, double tol, int maxit, double timeout_s) {
    char *ws = (char *)plan->d_work;
    const int n = plan->n_systems;
    const Fixed F = fixed_offsets(n, plan->max_blocks);
    BatchArgs a;
    a.sys = (const BatchSysDev *)(ws + F.sys);
    a.chunks = (const BatchChunkDev *)(ws + F.chunks);
    a.n_sys = n;
    a.n_chunks = plan->n_chunks;
    a.part = (double *)(ws + F.part);
    a.first_sys_of = (int *)(ws + F.fsys);
    a.ctrl = (CgCtrl *)ws;
    a.out_status = (int *)(ws + F.out_int);
    a.out_iters = a.out_status + n;
    a.out_rr = (double *)(ws + F.out_dbl);
    a.out_bb = a.out_rr + n;
    a.tol2 = tol * tol;
    a.maxit = maxit;
    a.max_blocks = plan->max_blocks;
    a.timeout_ns = (long long)((timeout_s > 0.0 ? timeout_s : 2.0) * 1e9);
    return a;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_cg_batched_workspace(int n_systems, const fe_matrix *A, size_t *h_bytes) {
    if (n_systems < 1 || n_systems > kBatchMaxSystems || !A || !h_bytes) return FE_ERR_ARG;
    for (int i = 0; i < n_systems; ++i) {
        fe_status st = check_matrix(&A[i]);
        if (st != FE_OK) return st;
    }
    *h_bytes = vector_offsets(n_systems, A, kCgMaxBlocks, nullptr);
    return FE_OK;
}

fe_status fe_cg_batched_plan(int n_systems, const fe_matrix *A, const double *const *d_b,
                             double *const *d_x, int krhs, int method, int blocks_per_sm, void *d_work,
                             size_t work_bytes, fe_batch_plan *h_plan, fe_stream_t stream) {
    if (n_systems < 1 || n_systems > kBatchMaxSystems || !A || !d_b || !d_x || !d_work || !h_plan)
        return FE_ERR_ARG;
    if (krhs != 1 && krhs != 2 && krhs != 4) return FE_ERR_ARG;
    if (method != FE_BATCH_TEXTBOOK && method != FE_BATCH_SINGLE_REDUCTION) return FE_ERR_ARG;
    if (!aligned(d_work, 256)) return FE_ERR_ARG;
    const int fmt = A[0].format;
    if (fmt != FE_FMT_BCRS3 && fmt != FE_FMT_SELL) return FE_ERR_ARG;
    for (int i = 0; i < n_systems; ++i) {
        fe_status st = check_matrix(&A[i]);
        if (st != FE_OK) return st;
        if (A[i].format != fmt || A[i].value_type != FE_VAL_F64 || A[i].n_rows != A[i].n_cols)
            return FE_ERR_ARG;
        if (!d_b[i] || !d_x[i] || !aligned(d_b[i], 8) || !aligned(d_x[i], 16)) return FE_ERR_ARG;
    }
    size_t need = 0;
    fe_status st = fe_cg_batched_workspace(n_systems, A, &need);
    if (st != FE_OK) return st;
    if (work_bytes < need) return FE_ERR_WORKSPACE;

    // groups: systems whose matrices are the same arrays, in first-seen order;
    // systems are renumbered group by group, chunks of krhs inside a group
    std::vector<int> group_of(n_systems, -1), order;
    std::vector<int> group_first;
    for (int i = 0; i < n_systems; ++i) {
        if (group_of[i] >= 0) continue;
        const int g = (int)group_first.size();
        group_first.push_back(i);
        for (int j = i; j < n_systems; ++j)
            if (group_of[j] < 0 && A[j].d_vals == A[i].d_vals && A[j].d_cols == A[i].d_cols &&
                A[j].d_slice_ptr == A[i].d_slice_ptr && A[j].n_rows == A[i].n_rows) {
                group_of[j] = g;
                order.push_back(j);
            }
    }
    std::vector<BatchChunkDev> chunks;
    std::vector<BatchSysDev> sys(n_systems);
    std::vector<int> slot_of(n_systems);   // caller's index -> position in the solve
    std::vector<size_t> voff;
    vector_offsets(n_systems, A, kCgMaxBlocks, &voff);
    const Fixed F = fixed_offsets(n_systems, kCgMaxBlocks);
    int pos = 0;
    for (size_t k = 0; k < order.size();) {
        const int g = group_of[order[k]];
        size_t e = k;
        while (e < order.size() && group_of[order[e]] == g) ++e;
        for (size_t c0 = k; c0 < e; c0 += krhs) {
            BatchChunkDev ch;
            ch.A = A[order[c0]];
            ch.first_sys = pos;
            ch.n_rhs = (int)std::min<size_t>(krhs, e - c0);
            ch.n_slices = (int)A[order[c0]].n_slices;
            ch.pad = 0;
            for (int j = 0; j < ch.n_rhs; ++j) {
                const int i = order[c0 + j];
                BatchSysDev &sd = sys[pos];
                char *base = (char *)d_work + voff[i];
                const size_t vb = align256((size_t)A[i].n_slices * kSlice * sizeof(double));
                sd.b = d_b[i];
                sd.x = d_x[i];
                sd.r = (double *)base;
                sd.p = (double *)(base + vb);
                sd.w = (double *)(base + 2 * vb);
                sd.s = (double *)(base + 3 * vb);
                sd.chunk = (int)chunks.size();
                sd.pad = i;   // caller's index
                slot_of[i] = pos;
                ++pos;
            }
            chunks.push_back(ch);
            k = c0 + ch.n_rhs;
        }
        k = e;
    }

    int per_sm = 0;
    const void *kern = batched_kernel(fmt, krhs, method);
    if (kern == nullptr) return FE_ERR_ARG;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, 0));
    if (per_sm < 1) return FE_ERR_CUDA;
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    long long total_slices = 0;
    for (const auto &ch : chunks) total_slices += ch.n_slices;
    long long grid = (long long)sm_count() * per_sm;
    const long long need_blocks = (total_slices + kCgWarps - 1) / kCgWarps;
    if (grid > need_blocks) grid = need_blocks;
    if (grid > kCgMaxBlocks) grid = kCgMaxBlocks;
    if (grid < 1) grid = 1;
    // A block's range never exceeds ceil(total / grid) units, whatever has
    // converged, so it spans at most that / (smallest chunk) + 2 chunks.
    {
        long long min_slices = total_slices;
        for (const auto &ch : chunks) min_slices = std::min<long long>(min_slices, ch.n_slices);
        const long long per_block = (total_slices + grid - 1) / grid;
        const long long span = per_block / std::max<long long>(min_slices, 1) + 2;
        if (span * krhs > kBatchMaxTouch) return FE_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    FE_TRY_CUDA(cudaMemcpyAsync((char *)d_work + F.sys, sys.data(), sizeof(BatchSysDev) * n_systems,
                                cudaMemcpyHostToDevice, s));
    FE_TRY_CUDA(cudaMemcpyAsync((char *)d_work + F.chunks, chunks.data(),
                                sizeof(BatchChunkDev) * chunks.size(), cudaMemcpyHostToDevice, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    h_plan->format = fmt;
    h_plan->krhs = krhs;
    h_plan->method = method;
    h_plan->n_systems = n_systems;
    h_plan->n_chunks = (int)chunks.size();
    h_plan->grid = (int)grid;
    h_plan->max_blocks = kCgMaxBlocks;
    h_plan->d_work = d_work;
    h_plan->work_bytes = work_bytes;
    for (int i = 0; i < n_systems && i < FE_BATCH_MAX_SYSTEMS; ++i) h_plan->slot_of[i] = slot_of[i];
    return FE_OK;
}

fe_status fe_cg_batched_launch(const fe_batch_plan *plan, double tol, int maxit, double timeout_s,
                               fe_stream_t stream) {
    if (!plan || !plan->d_work || maxit < 0 || !(tol >= 0.0) || plan->n_systems < 1 ||
        plan->n_systems > kBatchMaxSystems)
        return FE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BatchArgs a = args_of(plan, tol, maxit, timeout_s);
    const void *kern = batched_kernel(plan->format, plan->krhs, plan->method);
    if (kern == nullptr || plan->grid < 1 || plan->grid > plan->max_blocks) return FE_ERR_ARG;
    FE_TRY_CUDA(cudaMemsetAsync(a.ctrl, 0, sizeof(CgCtrl), s));
    void *params[] = {(void *)&a};
    FE_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3((unsigned)plan->grid), dim3(kBatchThreads), params, 0, s));
    return FE_OK;
}

fe_status fe_cg_batched_results(const fe_batch_plan *plan, fe_cg_result *h_results,
                                fe_stream_t stream) {
    if (!plan || !plan->d_work || !h_results) return FE_ERR_ARG;
    const int n = plan->n_systems;
    cudaStream_t s = (cudaStream_t)stream;
    BatchArgs a = args_of(plan, 0.0, 0, 0.0);
    std::vector<int> stat(n), it(n);
    std::vector<double> rr(n), bb(n);
    FE_TRY_CUDA(cudaMemcpyAsync(stat.data(), a.out_status, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaMemcpyAsync(it.data(), a.out_iters, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaMemcpyAsync(rr.data(), a.out_rr, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaMemcpyAsync(bb.data(), a.out_bb, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CgCtrl c;
    FE_TRY_CUDA(cudaMemcpyAsync(&c, a.ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    fe_status worst = FE_OK;
    for (int i = 0; i < n; ++i) {
        const int k = plan->slot_of[i];
        h_results[i].status = stat[k];
        h_results[i].iterations = it[k];
        h_results[i].bnorm = sqrt(bb[k]);
        h_results[i].relres = bb[k] > 0.0 ? sqrt(rr[k] / bb[k]) : 0.0;
        if (stat[k] != FE_OK && worst == FE_OK) worst = (fe_status)stat[k];
    }
    if (c.status != FE_OK) worst = (fe_status)c.status;
    return worst;
}

fe_status fe_cg_solve_batched(int n_systems, const fe_matrix *A, const double *const *d_b,
                              double *const *d_x, double tol, int maxit, int krhs, double timeout_s,
                              void *d_work, size_t work_bytes, fe_cg_result *h_results,
                              fe_stream_t stream) {
    fe_batch_plan plan;
    fe_status st = fe_cg_batched_plan(n_systems, A, d_b, d_x, krhs, FE_BATCH_TEXTBOOK, 0, d_work,
                                      work_bytes, &plan, stream);
    if (st != FE_OK) return st;
    st = fe_cg_batched_launch(&plan, tol, maxit, timeout_s, stream);
    if (st != FE_OK) return st;
    return fe_cg_batched_results(&plan, h_results, stream);
}

}  // extern "C"
