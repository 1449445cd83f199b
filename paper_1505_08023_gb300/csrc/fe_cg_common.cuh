// fe_cg_common.cuh -- pieces shared by the persistent CG kernels: the bounded
// grid barrier, the fixed-order grid reduction, the 16-byte streaming vector
// updates, and the residual kernels.
#pragma once

#include <math.h>

#include "fe_common.cuh"

namespace fe {

constexpr int kCgWarps = 8;
constexpr int kCgThreads = kCgWarps * 32;
constexpr int kCgMaxBlocks = 4096;
constexpr int kCgBlocksPerSm = 4;
// Resident blocks the persistent kernels are compiled for: the CSR slice
// kernel keeps seven entries per lane in flight, which needs more than the
// 64 registers of four blocks per SM.
template <int FMT> constexpr int cg_min_blocks() {
    return (FMT == FE_FMT_CSR || FMT == FE_FMT_VBCRS) ? 3 : kCgBlocksPerSm;
}
// The streaming CG kernels' BCRS3 SpMV issues the loads of all nine slots of
// a 27-point row in one trip and runs three blocks per SM (80 registers, no
// spills; four blocks at 64 registers spill): 1 % less time per step at
// N = 256 than three slots per trip at four blocks per SM.  The three- and
// two-phase kernels run the same block count, so both split the slices and
// the dot products the same way (their results are bitwise equal).
template <int FMT> constexpr int k_cg_unroll() { return FMT == FE_FMT_BCRS3 ? 9 : 0; }
template <int FMT> constexpr int k_cg_min_blocks() { return FMT == FE_FMT_BCRS3 ? 3 : cg_min_blocks<FMT>(); }
constexpr unsigned kMaxPolls = 1u << 28;

struct CgCtrl {
    unsigned long long bar;  // barrier arrivals
    int abort;               // set by a block whose wait timed out
    int status;              // fe_status of the solve
    int iterations;
    int pad;
    double rr;
    double bb;
};

template <class XT> struct CgArgs {
    fe_matrix A;
    const XT *b;
    XT *x, *r, *p, *w;
    double *part;            // [2][2 * kCgMaxBlocks]
    CgCtrl *ctrl;
    double tol2;
    int maxit;
    int x0_zero;             // start from x = 0 without reading x (skips one SpMV)
    long long timeout_ns;
    long long stall_barrier;  // fault injection: block 0 skips this arrival (-1: none)
    double *x64;             // if set: x64 += x on exit (mixed-precision refinement step)
    XT *p2;                  // second p buffer of the two-phase form (k_cg2)
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// State every thread of a block shares (identical in all of them): kept in
// shared memory so that the SpMV phase has the registers to itself.
struct CgBlockState {
    unsigned long long target;  // barrier arrivals this block waits for
    double rr, bb;              // r.r of the current step, b.b
    double red[kCgWarps][2];    // per-warp partials of the block reduction
    double sum[2];              // grid sums of the last reduction (read by all threads)
    int round;                  // reductions done (selects the partial buffer)
    int k;                      // CG steps done
    int ok;                     // 0 once a barrier wait gave up
};

// Grid barrier with a bounded wait.  Returns true (uniformly in the block) if
// all blocks arrived and nobody aborted.  SYNC_FIRST = false for a caller whose
// block is already synchronised and whose only work since is thread 0's.
template <bool SYNC_FIRST = true>
__device__ __forceinline__ bool grid_barrier(CgCtrl *ctrl, CgBlockState *st, long long timeout_ns,
                                             long long stall_barrier) {
    if (SYNC_FIRST) __syncthreads();
    if (threadIdx.x == 0) {
        const long long index = (long long)(st->target / gridDim.x);  // barriers passed so far
        const unsigned long long target = st->target + gridDim.x;
        st->target = target;
        int ok = 1;
        if (!(blockIdx.x == 0 && index == stall_barrier)) red_release_add(&ctrl->bar, 1ull);
        const long long t0 = global_ns();
        unsigned polls = 0;
        // one load in flight per poll; the abort flag and the clock every 8th
        // poll.  The acquire load that sees the count orders what the block
        // reads after the __syncthreads below (partials by ld.global.cg, the
        // gathers after the acquire has invalidated L1), so no fence follows.
        // A block that gave up has already arrived here; the others see its
        // abort flag at their next barrier and leave too (bounded either way).
        while (ld_acquire(&ctrl->bar) < target) {
            if (((++polls) & 7u) == 0) {
                if (*(volatile int *)&ctrl->abort) { ok = 0; break; }
                if (global_ns() - t0 > timeout_ns || polls > kMaxPolls) {
                    atomicExch(&ctrl->abort, 1);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        st->ok = ok;
    }
    __syncthreads();
    return st->ok != 0;
}

// Sum (v0, v1) over the whole grid: warp butterfly, fixed warp order, one
// 16-byte partial per block; after the barrier warp 0 of every block sums the
// partials in a fixed order (lane-strided, then a butterfly) and shares the
// result through shared memory.  One reading warp per block keeps the number
// of requests to the hot partial lines at G per block instead of 8 G.
// `a` is any argument block with part, ctrl, timeout_ns and stall_barrier.
template <class Args, bool TWO = true, int DIV = 0>
__device__ __forceinline__ bool grid_sum2(const Args &a, CgBlockState *st, double v0,
                                          double v1, double &o0, double &o1, double x = 0.0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v0 = warp_sum(v0);
    if (TWO) v1 = warp_sum(v1);
    if (lane == 0) {
        st->red[warp][0] = v0;
        st->red[warp][1] = TWO ? v1 : 0.0;
    }
    __syncthreads();
    double2 *part = reinterpret_cast<double2 *>(a.part + (size_t)(st->round & 1) * 2 * kCgMaxBlocks);
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
#pragma unroll
        for (int k = 0; k < kCgWarps; ++k) {
            t0 += st->red[k][0];
            t1 += st->red[k][1];
        }
        __stcg(part + blockIdx.x, make_double2(t0, t1));
    }
    // the __syncthreads above orders every thread's read of st->sum from the
    // previous reduction before warp 0 overwrites it below, and since then only
    // thread 0 has worked, so the barrier needs no block barrier of its own
    if (!grid_barrier<false>(a.ctrl, st, a.timeout_ns, a.stall_barrier)) return false;
    if (warp == 0) {
        // lane-strided partials, four loads in flight per lane (a loop of one
        // dependent load per trip costs an L2 round trip per 32 blocks); the
        // additions keep the order i, i + 32, i + 64, ...
        double t0 = 0.0, t1 = 0.0;
        const unsigned G = gridDim.x;
        for (unsigned i = lane; i < G; i += 128) {
            double2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = (i + 32 * u < G) ? __ldcg(part + i + 32 * u) : make_double2(0.0, 0.0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i + 32 * u < G) {
                    t0 += v[u].x;
                    if (TWO) t1 += v[u].y;
                }
            }
        }
        t0 = warp_sum(t0);
        if (TWO) t1 = warp_sum(t1);
        if (lane == 0) {
            st->sum[0] = t0;
            st->sum[1] = DIV == 1 ? x / t0 : (DIV == 2 ? t0 / x : t1);
            st->round += 1;            // every thread read st->round before the barrier
        }
    }
    __syncthreads();
    o0 = st->sum[0];
    o1 = st->sum[1];
    return true;
}

// One value: grid_sum2 without the second sum's shuffles.
template <class Args>
__device__ __forceinline__ bool grid_sum1(const Args &a, CgBlockState *st, double v0, double &o0) {
    double unused;
    return grid_sum2<Args, false>(a, st, v0, 0.0, o0, unused);
}

// One value and a quotient with it: x / sum (DIV = 1) or sum / x (DIV = 2),
// formed once per block by the warp that finishes the sum and published with
// it, so the other warps spend no FP64 division (each warp-wide FP64
// instruction costs the SM 16 cycles of its 2-per-clock FP64 pipe).
template <int DIV, class Args>
__device__ __forceinline__ bool grid_sum1_div(const Args &a, CgBlockState *st, double v0, double x, double &sum,
                                              double &quot) {
    return grid_sum2<Args, false, DIV>(a, st, v0, 0.0, sum, quot, x);
}

// 16-byte packs of the vector phases: the streaming passes (x, r update and
// p update) are bracketed by grid barriers, so they need not follow the
// SpMV's slice ownership; each thread moves two 16-byte packs per array per
// trip, which keeps enough bytes in flight to stream at HBM rate.
template <class XT> struct Pack16;
template <> struct Pack16<double> { using T = double2; static constexpr int N = 2; };
template <> struct Pack16<float> { using T = float4; static constexpr int N = 4; };

template <class XT> __device__ __forceinline__ XT &lane_of(typename Pack16<XT>::T &v, int i) {
    return reinterpret_cast<XT *>(&v)[i];
}

// The vectors below are rewritten by other blocks between grid barriers: no
// __restrict__, so every load stays on the coherent path.
// B: x += alpha p, r -= alpha w; returns this thread's partial of r.r
template <class XT>
__device__ __forceinline__ XT update_xr(XT *x, XT *r, const XT *p, const XT *w,
                                        int64_t m, XT alpha) {
    using P = typename Pack16<XT>::T;
    constexpr int V = Pack16<XT>::N;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t npk = m / V;
    P *x4 = reinterpret_cast<P *>(x), *r4 = reinterpret_cast<P *>(r);
    const P *p4 = reinterpret_cast<const P *>(p), *w4 = reinterpret_cast<const P *>(w);
    XT acc = XT(0);
    for (int64_t q = tid; q < npk; q += 2 * nth) {
        const int64_t q1 = q + nth;
        const bool two = q1 < npk;
        P xv[2], rv[2], pv[2], wv[2];
        xv[0] = x4[q]; rv[0] = r4[q]; pv[0] = p4[q]; wv[0] = w4[q];
        if (two) { xv[1] = x4[q1]; rv[1] = r4[q1]; pv[1] = p4[q1]; wv[1] = w4[q1]; }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                lane_of<XT>(xv[u], i) = fma(alpha, lane_of<XT>(pv[u], i), lane_of<XT>(xv[u], i));
                const XT ri = fma(-alpha, lane_of<XT>(wv[u], i), lane_of<XT>(rv[u], i));
                lane_of<XT>(rv[u], i) = ri;
                acc = fma(ri, ri, acc);
            }
        }
        x4[q] = xv[0]; r4[q] = rv[0];
        if (two) { x4[q1] = xv[1]; r4[q1] = rv[1]; }
    }
    for (int64_t row = npk * V + tid; row < m; row += nth) {
        x[row] = fma(alpha, p[row], x[row]);
        const XT ri = fma(-alpha, w[row], r[row]);
        r[row] = ri;
        acc = fma(ri, ri, acc);
    }
    return acc;
}

// B of k_cg: r -= alpha w; returns this thread's partial of r.r (x waits for C)
template <class XT>
__device__ __forceinline__ XT update_r(XT *r, const XT *w, int64_t m, XT alpha) {
    using P = typename Pack16<XT>::T;
    constexpr int V = Pack16<XT>::N;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t npk = m / V;
    P *r4 = reinterpret_cast<P *>(r);
    const P *w4 = reinterpret_cast<const P *>(w);
    XT acc = XT(0);
    for (int64_t q = tid; q < npk; q += 2 * nth) {
        const int64_t q1 = q + nth;
        const bool two = q1 < npk;
        P rv[2], wv[2];
        rv[0] = r4[q]; wv[0] = w4[q];
        if (two) { rv[1] = r4[q1]; wv[1] = w4[q1]; }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const XT ri = fma(-alpha, lane_of<XT>(wv[u], i), lane_of<XT>(rv[u], i));
                lane_of<XT>(rv[u], i) = ri;
                acc = fma(ri, ri, acc);
            }
        }
        r4[q] = rv[0];
        if (two) r4[q1] = rv[1];
    }
    for (int64_t row = npk * V + tid; row < m; row += nth) {
        const XT ri = fma(-alpha, w[row], r[row]);
        r[row] = ri;
        acc = fma(ri, ri, acc);
    }
    return acc;
}

// C of k_cg: x += alpha p with the step's old p, then p = r + beta p
template <class XT>
__device__ __forceinline__ void update_xp(XT *x, XT *p, const XT *r, int64_t m, XT alpha, XT beta) {
    using P = typename Pack16<XT>::T;
    constexpr int V = Pack16<XT>::N;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t npk = m / V;
    P *x4 = reinterpret_cast<P *>(x), *p4 = reinterpret_cast<P *>(p);
    const P *r4 = reinterpret_cast<const P *>(r);
    for (int64_t q = tid; q < npk; q += 2 * nth) {
        const int64_t q1 = q + nth;
        const bool two = q1 < npk;
        P xv[2], pv[2], rv[2];
        xv[0] = x4[q]; pv[0] = p4[q]; rv[0] = r4[q];
        if (two) { xv[1] = x4[q1]; pv[1] = p4[q1]; rv[1] = r4[q1]; }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const XT pi = lane_of<XT>(pv[u], i);
                lane_of<XT>(xv[u], i) = fma(alpha, pi, lane_of<XT>(xv[u], i));
                lane_of<XT>(pv[u], i) = fma(beta, pi, lane_of<XT>(rv[u], i));
            }
        }
        x4[q] = xv[0]; p4[q] = pv[0];
        if (two) { x4[q1] = xv[1]; p4[q1] = pv[1]; }
    }
    for (int64_t row = npk * V + tid; row < m; row += nth) {
        const XT pi = p[row];
        x[row] = fma(alpha, pi, x[row]);
        p[row] = fma(beta, pi, r[row]);
    }
}

// C: p = r + beta p
template <class XT>
__device__ __forceinline__ void update_p(XT *p, const XT *r, int64_t m,
                                         XT beta) {
    using P = typename Pack16<XT>::T;
    constexpr int V = Pack16<XT>::N;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t npk = m / V;
    P *p4 = reinterpret_cast<P *>(p);
    const P *r4 = reinterpret_cast<const P *>(r);
    for (int64_t q = tid; q < npk; q += 2 * nth) {
        const int64_t q1 = q + nth;
        const bool two = q1 < npk;
        P pv[2], rv[2];
        pv[0] = p4[q]; rv[0] = r4[q];
        if (two) { pv[1] = p4[q1]; rv[1] = r4[q1]; }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            lane_of<XT>(pv[0], i) = fma(beta, lane_of<XT>(pv[0], i), lane_of<XT>(rv[0], i));
            lane_of<XT>(pv[1], i) = fma(beta, lane_of<XT>(pv[1], i), lane_of<XT>(rv[1], i));
        }
        p4[q] = pv[0];
        if (two) p4[q1] = pv[1];
    }
    for (int64_t row = npk * V + tid; row < m; row += nth) p[row] = fma(beta, p[row], r[row]);
}

// r = b - A x over the block's slices; r.r and b.b partials per block.
// With r32 set, also stores r in FP32 (the right-hand side of the inner solve
// of the mixed-precision form).
template <int FMT, class VT>
__global__ void __launch_bounds__(kCgThreads) k_resid(const fe_matrix A, const double *__restrict__ b,
                                                      const double *__restrict__ x,
                                                      double *__restrict__ part,
                                                      float *__restrict__ r32) {
    __shared__ double red[kCgWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s0 = 0.0, s1 = 0.0;
    const int64_t tw = (int64_t)gridDim.x * kCgWarps;
    for (int64_t s = (int64_t)blockIdx.x * kCgWarps + warp; s < A.n_slices; s += tw) {
        const double ax = slice_spmv<FMT, VT, double, double, true>(A, s, lane, x);
        const int64_t row = s * kSlice + lane;
        if (row < A.n_rows) {
            const double bi = b[row], ri = bi - ax;
            if (r32 != nullptr) r32[row] = (float)ri;
            s0 = fma(ri, ri, s0);
            s1 = fma(bi, bi, s1);
        }
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (lane == 0) {
        red[warp][0] = s0;
        red[warp][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int k = 0; k < kCgWarps; ++k) {
            t0 += red[k][0];
            t1 += red[k][1];
        }
        part[2 * blockIdx.x] = t0;
        part[2 * blockIdx.x + 1] = t1;
    }
}

static __global__ void k_resid_final(int nblocks, const double *__restrict__ part, double *__restrict__ out) {
    const int lane = threadIdx.x;
    double t0 = 0.0, t1 = 0.0;
    for (int i = lane; i < nblocks; i += 32) {
        t0 += part[2 * i];
        t1 += part[2 * i + 1];
    }
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    if (lane == 0) {
        out[0] = t0;
        out[1] = t1;
    }
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

template <int FMT, class VT>
static fe_status launch_resid(const fe_matrix &A, const double *b, const double *x, double *part,
                              float *r32, int *nblocks, cudaStream_t s) {
    auto kern = k_resid<FMT, VT>;
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (A.n_slices + kCgWarps - 1) / kCgWarps;
    if (blocks > need) blocks = need;
    if (blocks > kCgMaxBlocks) blocks = kCgMaxBlocks;
    if (blocks < 1) blocks = 1;
    kern<<<(int)blocks, kCgThreads, 0, s>>>(A, b, x, part, r32);
    FE_TRY_LAUNCH();
    *nblocks = (int)blocks;
    return FE_OK;
}

#define FE_DISPATCH_FMT_VT(A, FN, ...)                                                     \
    switch ((A).format * 3 + (A).value_type) {                                             \
        case FE_FMT_CSR * 3 + FE_VAL_F64: return FN<FE_FMT_CSR, double>(__VA_ARGS__);       \
        case FE_FMT_CSR * 3 + FE_VAL_F32: return FN<FE_FMT_CSR, float>(__VA_ARGS__);        \
        case FE_FMT_CSR * 3 + FE_VAL_BF16: return FN<FE_FMT_CSR, __nv_bfloat16>(__VA_ARGS__); \
        case FE_FMT_SELL * 3 + FE_VAL_F64: return FN<FE_FMT_SELL, double>(__VA_ARGS__);     \
        case FE_FMT_SELL * 3 + FE_VAL_F32: return FN<FE_FMT_SELL, float>(__VA_ARGS__);      \
        case FE_FMT_SELL * 3 + FE_VAL_BF16: return FN<FE_FMT_SELL, __nv_bfloat16>(__VA_ARGS__); \
        case FE_FMT_BCRS3 * 3 + FE_VAL_F64: return FN<FE_FMT_BCRS3, double>(__VA_ARGS__);   \
        case FE_FMT_BCRS3 * 3 + FE_VAL_F32: return FN<FE_FMT_BCRS3, float>(__VA_ARGS__);    \
        case FE_FMT_BCRS3 * 3 + FE_VAL_BF16: return FN<FE_FMT_BCRS3, __nv_bfloat16>(__VA_ARGS__); \
        case FE_FMT_VBCRS * 3 + FE_VAL_F64: return FN<FE_FMT_VBCRS, double>(__VA_ARGS__);   \
        case FE_FMT_VBCRS * 3 + FE_VAL_F32: return FN<FE_FMT_VBCRS, float>(__VA_ARGS__);    \
        case FE_FMT_VBCRS * 3 + FE_VAL_BF16: return FN<FE_FMT_VBCRS, __nv_bfloat16>(__VA_ARGS__); \
        default: return FE_ERR_ARG;                                                        \
    }

static inline fe_status dispatch_resid(const fe_matrix &A, const double *b, const double *x, double *part,
                                float *r32, int *nblocks, cudaStream_t s) {
    FE_DISPATCH_FMT_VT(A, launch_resid, A, b, x, part, r32, nblocks, s)
}


// Launch of the FP32-vector CG kernel (defined in fe_cg.cu): the inner solver
// of the restarted mixed-precision mode.
fe_status launch_cg_f32(const CgArgs<float> &args, cudaStream_t s);

// The matrix-resident CG kernel (fe_cg_resident.cu): whether A qualifies (FP64
// BCRS3 or sliced-ELL values, at most one slice per warp of one block per SM),
// and its launch; *taken is false when the grid would not be co-resident.
bool resident_cg_fits(const fe_matrix &A);
fe_status launch_cg_resident(const CgArgs<double> &args, cudaStream_t s, bool *taken);

// Barrier index armed by fe_inject_barrier_stall (test hook), consumed by the
// next solve that takes it (-1: none).  Defined in fe_cg.cu.
long long take_stall_barrier();

}  // namespace fe
