// fe_cg.cu -- unpreconditioned CG (paper Sec. 1: MATVEC + DOT + WAXPY) as
// one persistent cooperative kernel per solve, and the true-residual check.
//
// Each CG step is three phases separated by grid barriers:
//   A  w = A p over the block's slices, p.w accumulated in the SpMV epilogue
//   B  x += alpha p, r -= alpha w, r.r accumulated in the same pass
//   C  p = r + beta p
// A dot product is reduced warp (xor butterfly) -> block (fixed warp order)
// -> one partial per block in global memory -> after the barrier every warp
// of every block sums the partials in block order, so all blocks hold the
// same bits and take the same branch, and a rerun reproduces every bit.
// Two partial buffers alternate, so a block that races ahead into the next
// reduction never overwrites partials another block is still reading.
//
// The same kernel, instantiated with FP32 vectors, is the inner solver of the
// mixed-precision form: SpMV and per-thread dot partials in FP32, the grid
// reduction of every dot product in FP64, alpha and beta in FP64.
//
// The grid barrier counts arrivals on a 64-bit counter (release add, acquire
// poll).  Every wait is bounded: past `timeout_ns` (or a poll cap) the block
// raises the abort flag and leaves; the others see the flag at their next
// wait and leave too, and the host reports FE_ERR_TIMEOUT.  Nothing traps.
#include <math.h>

#include <mutex>

#include "fe_common.cuh"

namespace fe {

constexpr int kCgWarps = 8;
constexpr int kCgThreads = kCgWarps * 32;
constexpr int kCgMaxBlocks = 4096;
constexpr int kCgBlocksPerSm = 4;
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
    int round;                  // reductions done (selects the partial buffer)
    int k;                      // CG steps done
    int ok;                     // 0 once a barrier wait gave up
};

// Grid barrier with a bounded wait.  Returns true (uniformly in the block) if
// all blocks arrived and nobody aborted.
__device__ __forceinline__ bool grid_barrier(CgCtrl *ctrl, CgBlockState *st, long long timeout_ns,
                                             long long stall_barrier) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long index = (long long)(st->target / gridDim.x);  // barriers passed so far
        const unsigned long long target = st->target + gridDim.x;
        st->target = target;
        int ok = 1;
        if (!(blockIdx.x == 0 && index == stall_barrier)) red_release_add(&ctrl->bar, 1ull);
        const long long t0 = global_ns();
        unsigned polls = 0;
        while (ld_acquire(&ctrl->bar) < target) {
            if (*(volatile int *)&ctrl->abort) { ok = 0; break; }
            if (((++polls) & 7u) == 0 &&
                (global_ns() - t0 > timeout_ns || polls > kMaxPolls)) {
                atomicExch(&ctrl->abort, 1);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        if (ok && *(volatile int *)&ctrl->abort) ok = 0;
        __threadfence();
        st->ok = ok;
    }
    __syncthreads();
    return st->ok != 0;
}

// Sum (v0, v1) over the whole grid; see the file comment for the order.
template <class XT>
__device__ __forceinline__ bool grid_sum2(const CgArgs<XT> &a, CgBlockState *st, double v0,
                                          double v1, double &o0, double &o1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
        st->red[warp][0] = v0;
        st->red[warp][1] = v1;
    }
    __syncthreads();
    double *part = a.part + (size_t)(st->round & 1) * 2 * kCgMaxBlocks;
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
#pragma unroll
        for (int k = 0; k < kCgWarps; ++k) {
            t0 += st->red[k][0];
            t1 += st->red[k][1];
        }
        __stcg(part + 2 * blockIdx.x, t0);
        __stcg(part + 2 * blockIdx.x + 1, t1);
    }
    if (!grid_barrier(a.ctrl, st, a.timeout_ns, a.stall_barrier)) return false;
    double t0 = 0.0, t1 = 0.0;
    for (unsigned i = lane; i < gridDim.x; i += 32) {
        t0 += __ldcg(part + 2 * i);
        t1 += __ldcg(part + 2 * i + 1);
    }
    o0 = warp_sum(t0);
    o1 = warp_sum(t1);
    __syncthreads();                       // every warp has read st->round
    if (threadIdx.x == 0) st->round += 1;
    return true;
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

// B: x += alpha p, r -= alpha w; returns this thread's partial of r.r
template <class XT>
__device__ __forceinline__ XT update_xr(XT *__restrict__ x, XT *__restrict__ r,
                                        const XT *__restrict__ p, const XT *__restrict__ w,
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

// C: p = r + beta p
template <class XT>
__device__ __forceinline__ void update_p(XT *__restrict__ p, const XT *__restrict__ r, int64_t m,
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

template <int FMT, class VT, class XT>
__global__ void __launch_bounds__(kCgThreads, kCgBlocksPerSm) k_cg(const CgArgs<XT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ CgBlockState st;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    XT *sv = reinterpret_cast<XT *>(smem_raw) + (size_t)warp * 2 * kCsrStage;
    XT *sx = sv + kCsrStage;
    // rows fit int32 (check_matrix); slices are walked in a grid-stride order
    const int m = (int)a.A.n_rows, ns = (int)a.A.n_slices;
    const int tw = gridDim.x * kCgWarps;
    if (threadIdx.x == 0) {
        st.target = 0;
        st.round = 0;
        st.k = 0;
        st.ok = 1;
    }
    __syncthreads();
    int status = FE_ERR_MAXIT;
    bool alive = true;

    // r = b - A x, p = r; r.r and b.b
    {
        XT s0 = XT(0), s1 = XT(0);
        for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
            XT ax = XT(0);
            if (!a.x0_zero) ax = slice_spmv<FMT, VT, XT, XT, false>(a.A, s, lane, a.x, sv, sx);
            const int row = s * kSlice + lane;
            if (row < m) {
                const XT bi = a.b[row];
                const XT ri = bi - ax;
                if (a.x0_zero) a.x[row] = XT(0);
                a.r[row] = ri;
                a.p[row] = ri;
                s0 = fma(ri, ri, s0);
                s1 = fma(bi, bi, s1);
            }
        }
        double rr0, bb0;
        alive = grid_sum2(a, &st, (double)s0, (double)s1, rr0, bb0);
        if (threadIdx.x == 0) {
            st.rr = rr0;
            st.bb = bb0;
        }
        __syncthreads();
    }
    if (alive && st.bb == 0.0) {  // b = 0: the solution is 0
        for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
            const int row = s * kSlice + lane;
            if (row < m) a.x[row] = XT(0);
        }
        if (threadIdx.x == 0) st.rr = 0.0;
        status = FE_OK;
    } else {
        while (alive) {
            if (st.rr <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
            // A: w = A p, p.w
            XT pw_part = XT(0);
            for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
                const XT y = slice_spmv<FMT, VT, XT, XT, false>(a.A, s, lane, a.p, sv, sx);
                const int row = s * kSlice + lane;
                if (row < m) {
                    a.w[row] = y;
                    pw_part = fma(a.p[row], y, pw_part);
                }
            }
            double pw, unused;
            if (!(alive = grid_sum2(a, &st, (double)pw_part, 0.0, pw, unused))) break;
            if (!(pw > 0.0) || !(pw < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            // B: x += alpha p, r -= alpha w, r.r
            const XT rr_part = update_xr<XT>(a.x, a.r, a.p, a.w, m, (XT)(st.rr / pw));
            double rr_new;
            if (!(alive = grid_sum2(a, &st, (double)rr_part, 0.0, rr_new, unused))) break;
            const double beta = rr_new / st.rr;
            __syncthreads();                 // every thread has read st.rr
            if (threadIdx.x == 0) {
                st.rr = rr_new;
                st.k += 1;
            }
            __syncthreads();
            if (rr_new <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
            // C: p = r + beta p
            update_p<XT>(a.p, a.r, m, (XT)beta);
            if (!(alive = grid_barrier(a.ctrl, &st, a.timeout_ns, a.stall_barrier))) break;
        }
    }
    // refinement step of the mixed-precision form: x64 += x
    if (a.x64 != nullptr && alive && (status == FE_OK || status == FE_ERR_MAXIT)) {
        const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
        for (int row = tid; row < m; row += nth) a.x64[row] += (double)a.x[row];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = st.k;
        a.ctrl->rr = st.rr;
        a.ctrl->bb = st.bb;
    }
}

// r = b - A x over the block's slices; r.r and b.b partials per block.
// With r32 set, also stores r in FP32 (the right-hand side of the inner solve
// of the mixed-precision form).
template <int FMT, class VT>
__global__ void __launch_bounds__(kCgThreads) k_resid(const fe_matrix A, const double *__restrict__ b,
                                                      const double *__restrict__ x,
                                                      double *__restrict__ part,
                                                      float *__restrict__ r32) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kCgWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *sv = reinterpret_cast<double *>(smem_raw) + (size_t)warp * 2 * kCsrStage;
    double *sx = sv + kCsrStage;
    double s0 = 0.0, s1 = 0.0;
    const int64_t tw = (int64_t)gridDim.x * kCgWarps;
    for (int64_t s = (int64_t)blockIdx.x * kCgWarps + warp; s < A.n_slices; s += tw) {
        const double ax = slice_spmv<FMT, VT, double, double, true>(A, s, lane, x, sv, sx);
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

__global__ void k_resid_final(int nblocks, const double *__restrict__ part, double *__restrict__ out) {
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

static thread_local long long g_stall_barrier = -1;

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

static size_t cg_workspace_bytes(const fe_matrix &A) {
    const size_t vec = align256((size_t)A.n_slices * kSlice * sizeof(double));
    return 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) + 3 * vec;
}

template <int FMT, class VT, class XT>
static fe_status launch_cg(const CgArgs<XT> &args, cudaStream_t s) {
    auto kern = k_cg<FMT, VT, XT>;
    const size_t smem = spmv_smem_bytes<FMT, XT>(kCgWarps);
    if (smem > 48 * 1024)
        FE_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, smem));
    if (per_sm < 1) return FE_ERR_CUDA;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (args.A.n_slices + kCgWarps - 1) / kCgWarps;
    if (blocks > need) blocks = need;
    if (blocks > kCgMaxBlocks) blocks = kCgMaxBlocks;
    if (blocks < 1) blocks = 1;
    void *params[] = {(void *)&args};
    FE_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)blocks), dim3(kCgThreads),
                                            params, smem, s));
    return FE_OK;
}

template <int FMT, class VT>
static fe_status launch_resid(const fe_matrix &A, const double *b, const double *x, double *part,
                              float *r32, int *nblocks, cudaStream_t s) {
    auto kern = k_resid<FMT, VT>;
    const size_t smem = spmv_smem_bytes<FMT, double>(kCgWarps);
    if (smem > 48 * 1024)
        FE_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (A.n_slices + kCgWarps - 1) / kCgWarps;
    if (blocks > need) blocks = need;
    if (blocks > kCgMaxBlocks) blocks = kCgMaxBlocks;
    if (blocks < 1) blocks = 1;
    kern<<<(int)blocks, kCgThreads, smem, s>>>(A, b, x, part, r32);
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
        default: return FE_ERR_ARG;                                                        \
    }

template <int FMT, class VT> static fe_status launch_cg64(const CgArgs<double> &a, cudaStream_t s) {
    return launch_cg<FMT, VT, double>(a, s);
}
template <int FMT, class VT> static fe_status launch_cg32(const CgArgs<float> &a, cudaStream_t s) {
    return launch_cg<FMT, VT, float>(a, s);
}

static fe_status dispatch_cg(const CgArgs<double> &args, cudaStream_t s) {
    FE_DISPATCH_FMT_VT(args.A, launch_cg64, args, s)
}

static fe_status dispatch_cg(const CgArgs<float> &args, cudaStream_t s) {
    FE_DISPATCH_FMT_VT(args.A, launch_cg32, args, s)
}

static fe_status dispatch_resid(const fe_matrix &A, const double *b, const double *x, double *part,
                                float *r32, int *nblocks, cudaStream_t s) {
    FE_DISPATCH_FMT_VT(A, launch_resid, A, b, x, part, r32, nblocks, s)
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_inject_barrier_stall(int barrier_index) {
    if (barrier_index < -1) return FE_ERR_ARG;
    g_stall_barrier = barrier_index;
    return FE_OK;
}

fe_status fe_cg_workspace(const fe_matrix *A, size_t *h_bytes) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (h_bytes == nullptr) return FE_ERR_ARG;
    *h_bytes = cg_workspace_bytes(*A);
    return FE_OK;
}

fe_status fe_cg_solve(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                      double timeout_s, void *d_work, size_t work_bytes, fe_cg_result *h_result,
                      fe_stream_t stream) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (!d_b || !d_x || !d_work || !h_result || maxit < 0 || !(tol >= 0.0)) return FE_ERR_ARG;
    if (A->n_rows != A->n_cols) return FE_ERR_ARG;
    if (!aligned(d_b, 16) || !aligned(d_x, 16) || !aligned(d_work, 256)) return FE_ERR_ARG;
    if (work_bytes < cg_workspace_bytes(*A)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;

    char *ws = (char *)d_work;
    CgArgs<double> args;
    args.A = *A;
    args.b = d_b;
    args.x = d_x;
    args.ctrl = (CgCtrl *)ws;
    args.part = (double *)(ws + 256);
    const size_t vec = align256((size_t)A->n_slices * kSlice * sizeof(double));
    char *v0 = ws + 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double));
    args.r = (double *)v0;
    args.p = (double *)(v0 + vec);
    args.w = (double *)(v0 + 2 * vec);
    args.tol2 = tol * tol;
    args.maxit = maxit;
    const double tmo = timeout_s > 0.0 ? timeout_s : 2.0;
    args.timeout_ns = (long long)(tmo * 1e9);
    args.stall_barrier = g_stall_barrier;
    args.x0_zero = 0;
    args.x64 = nullptr;
    g_stall_barrier = -1;

    FE_TRY_CUDA(cudaMemsetAsync(args.ctrl, 0, sizeof(CgCtrl), s));
    st = dispatch_cg(args, s);
    if (st != FE_OK) return st;
    CgCtrl ctrl;
    FE_TRY_CUDA(cudaMemcpyAsync(&ctrl, args.ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    h_result->status = ctrl.status;
    h_result->iterations = ctrl.iterations;
    h_result->bnorm = sqrt(ctrl.bb);
    h_result->relres = ctrl.bb > 0.0 ? sqrt(ctrl.rr / ctrl.bb) : 0.0;
    return (fe_status)ctrl.status;
}

fe_status fe_true_relres(const fe_matrix *A, const double *d_b, const double *d_x, void *d_work,
                         size_t work_bytes, double *h_relres, fe_stream_t stream) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (!d_b || !d_x || !d_work || !h_relres || !aligned(d_work, 8)) return FE_ERR_ARG;
    if (work_bytes < FE_RESID_WORK_BYTES) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double *part = (double *)d_work;
    double *out = part + 2 * kCgMaxBlocks;
    int nblocks = 0;
    st = dispatch_resid(*A, d_b, d_x, part, nullptr, &nblocks, s);
    if (st != FE_OK) return st;
    k_resid_final<<<1, 32, 0, s>>>(nblocks, part, out);
    FE_TRY_LAUNCH();
    double h[2];
    FE_TRY_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    *h_relres = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
    return FE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- mixed precision

namespace fe {

static size_t mixed_workspace_bytes(const fe_matrix &lo) {
    const size_t vec = align256((size_t)lo.n_slices * kSlice * sizeof(float));
    return 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) +
           align256(FE_RESID_WORK_BYTES) + 5 * vec;
}

}  // namespace fe

extern "C" {

fe_status fe_cg_mixed_workspace(const fe_matrix *A_lo, size_t *h_bytes) {
    fe_status st = check_matrix(A_lo);
    if (st != FE_OK) return st;
    if (h_bytes == nullptr) return FE_ERR_ARG;
    *h_bytes = mixed_workspace_bytes(*A_lo);
    return FE_OK;
}

fe_status fe_cg_solve_mixed(const fe_matrix *A64, const fe_matrix *A_lo, const double *d_b,
                            double *d_x, double tol, int max_outer, double inner_tol,
                            int max_inner, double timeout_s, void *d_work, size_t work_bytes,
                            fe_mixed_result *h_result, fe_stream_t stream) {
    fe_status st = check_matrix(A64);
    if (st != FE_OK) return st;
    st = check_matrix(A_lo);
    if (st != FE_OK) return st;
    if (A64->value_type != FE_VAL_F64 || A64->n_rows != A64->n_cols ||
        A_lo->n_rows != A64->n_rows || A_lo->n_cols != A64->n_cols)
        return FE_ERR_ARG;
    if (!d_b || !d_x || !d_work || !h_result || max_outer < 0 || max_inner < 0 || !(tol >= 0.0) ||
        !(inner_tol > 0.0 && inner_tol < 1.0))
        return FE_ERR_ARG;
    if (!aligned(d_b, 8) || !aligned(d_x, 8) || !aligned(d_work, 256)) return FE_ERR_ARG;
    if (work_bytes < mixed_workspace_bytes(*A_lo)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;

    char *ws = (char *)d_work;
    CgCtrl *ctrl = (CgCtrl *)ws;
    double *cg_part = (double *)(ws + 256);
    char *q = ws + 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double));
    double *res_part = (double *)q;
    double *res_out = res_part + 2 * kCgMaxBlocks;
    q += align256(FE_RESID_WORK_BYTES);
    const size_t vec = align256((size_t)A_lo->n_slices * kSlice * sizeof(float));
    float *r32 = (float *)q, *d32 = (float *)(q + vec), *ri = (float *)(q + 2 * vec),
          *pi = (float *)(q + 3 * vec), *wi = (float *)(q + 4 * vec);

    CgArgs<float> in;
    in.A = *A_lo;
    in.b = r32;
    in.x = d32;
    in.r = ri;
    in.p = pi;
    in.w = wi;
    in.part = cg_part;
    in.ctrl = ctrl;
    in.tol2 = inner_tol * inner_tol;
    in.maxit = max_inner;
    in.x0_zero = 1;
    in.timeout_ns = (long long)((timeout_s > 0.0 ? timeout_s : 2.0) * 1e9);
    in.stall_barrier = -1;
    in.x64 = d_x;

    int outer = 0, inner_total = 0, status = FE_ERR_MAXIT;
    double relres = 0.0, bnorm = 0.0;
    while (true) {
        // r = b - A64 x in FP64 (stored in FP32 for the inner solve), ||r||, ||b||
        int nb = 0;
        st = dispatch_resid(*A64, d_b, d_x, res_part, r32, &nb, s);
        if (st != FE_OK) return st;
        k_resid_final<<<1, 32, 0, s>>>(nb, res_part, res_out);
        FE_TRY_LAUNCH();
        double h[2];
        FE_TRY_CUDA(cudaMemcpyAsync(h, res_out, sizeof(h), cudaMemcpyDeviceToHost, s));
        FE_TRY_CUDA(cudaStreamSynchronize(s));
        bnorm = sqrt(h[1]);
        if (h[1] == 0.0) {  // b = 0: the solution is 0
            FE_TRY_CUDA(cudaMemsetAsync(d_x, 0, (size_t)A64->n_rows * sizeof(double), s));
            FE_TRY_CUDA(cudaStreamSynchronize(s));
            relres = 0.0;
            status = FE_OK;
            break;
        }
        relres = sqrt(h[0] / h[1]);
        if (!(relres == relres)) { status = FE_ERR_BREAKDOWN; break; }
        if (relres <= tol) { status = FE_OK; break; }
        if (outer >= max_outer) { status = FE_ERR_MAXIT; break; }
        // inner FP32 CG on A_lo d = r, then x += d (inside the kernel)
        FE_TRY_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(CgCtrl), s));
        st = dispatch_cg(in, s);
        if (st != FE_OK) return st;
        CgCtrl c;
        FE_TRY_CUDA(cudaMemcpyAsync(&c, ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s));
        FE_TRY_CUDA(cudaStreamSynchronize(s));
        inner_total += c.iterations;
        ++outer;
        if (c.status == FE_ERR_TIMEOUT || c.status == FE_ERR_BREAKDOWN) { status = c.status; break; }
    }
    h_result->status = status;
    h_result->outer_iterations = outer;
    h_result->inner_iterations = inner_total;
    h_result->relres = relres;
    h_result->bnorm = bnorm;
    return (fe_status)status;
}

}  // extern "C"

// ---------------------------------------------------------------- solve without allocation
//
// fe_cg_solve_noalloc serves callers that cannot allocate device memory when
// they solve: code inside a latency-critical loop, where cudaMalloc's implicit
// device-wide synchronisation is not acceptable, or a plugin whose host
// framework owns every device buffer and forbids driver allocations.  They
// still pass A, b and x; the solver's own scratch (barrier/result block,
// reduction partials and the r, p, w vectors) lives in the file-scope array
// below, which every GPU that loads this library holds until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it.

namespace fe {

constexpr size_t kNoallocVecBytes = ((size_t)FE_NOALLOC_MAX_ROWS * sizeof(double) + 255) & ~(size_t)255;
constexpr size_t kNoallocBytes =
    256 + ((2 * 2 * (size_t)kCgMaxBlocks * sizeof(double) + 255) & ~(size_t)255) + 3 * kNoallocVecBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];

// Device address of g_noalloc_scratch on the current device (looked up once).
static fe_status noalloc_scratch(void **out) {
    int dev = 0;
    FE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FE_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *p = nullptr;
        FE_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return FE_OK;
}

}  // namespace fe

extern "C" {

fe_status fe_cg_solve_noalloc(const fe_matrix *A, const double *d_b, double *d_x, double tol,
                              int maxit, double timeout_s, fe_cg_result *h_result,
                              fe_stream_t stream) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (A->n_slices * (int64_t)kSlice > (int64_t)FE_NOALLOC_MAX_ROWS) return FE_ERR_WORKSPACE;
    const size_t need = cg_workspace_bytes(*A);
    if (need > kNoallocBytes) return FE_ERR_WORKSPACE;
    void *ws = nullptr;
    st = noalloc_scratch(&ws);
    if (st != FE_OK) return st;
    return fe_cg_solve(A, d_b, d_x, tol, maxit, timeout_s, ws, need, h_result, stream);
}

}  // extern "C"
