// fe_cg_sr.cu -- single-reduction CG (Chronopoulos and Gear, 1989: the s = 1
// member of their s-step family) as one persistent cooperative kernel.
//
// Same iterates as textbook CG in exact arithmetic, but a step needs one grid
// reduction instead of two, so it has two grid barriers instead of three:
//   U  p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s
//      (s carries A p by recurrence), then a barrier (the SpMV gathers r);
//   S  w = A r over the block's slices, with gamma = r.r and delta = w.r both
//      accumulated in the SpMV epilogue, then one fixed-order grid reduction
//      of the pair.
// The scalars follow from the reduced pair:
//   beta_k = gamma_k / gamma_{k-1},  p.Ap = delta_k - beta_k gamma_k / alpha_{k-1},
//   alpha_k = gamma_k / p.Ap          (k = 0: beta = 0, p.Ap = delta).
// In finite precision the curvature recurrence can lose its sign near
// convergence (cancellation); a step whose recurrence gives p.Ap <= 0 restarts
// the direction (beta = 0, p.Ap = delta = r.Ar) -- the oracle does the same --
// and only delta <= 0 is a breakdown.
// It pays off where barriers dominate the step (small meshes); on large
// meshes it moves the same bytes as textbook CG and does one more FMA per
// row (the s update), which matters on GB300's FP64 pipe.
// Reductions, barrier, timeout and determinism are those of k_cg
// (fe_cg_common.cuh).
#include "fe_cg_common.cuh"

namespace fe {

struct CgSrArgs : CgArgs<double> {
    double *s;  // A p, carried by its recurrence
};

// Block-uniform scalars of the recurrences (identical in every block).
struct SrState {
    double gamma, gamma_prev, delta, alpha_prev;
    double alpha, beta, curv;   // the step's scalars, formed once per block by thread 0
};

// U: p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s.  One 16-byte
// pack of each vector per thread per trip (five loads in flight per thread).
// No __restrict__: other blocks rewrite these vectors between barriers.
__device__ __forceinline__ void update_sr(double *x, double *r, double *p, double *s, const double *w,
                                          int64_t m, double alpha, double beta) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t npk = m / 2;
    double2 *x2 = reinterpret_cast<double2 *>(x), *r2 = reinterpret_cast<double2 *>(r);
    double2 *p2 = reinterpret_cast<double2 *>(p), *s2 = reinterpret_cast<double2 *>(s);
    const double2 *w2 = reinterpret_cast<const double2 *>(w);
    for (int64_t q = tid; q < npk; q += nth) {
        double2 xv = x2[q], rv = r2[q], pv = p2[q], sv = s2[q];
        const double2 wv = w2[q];
        pv.x = fma(beta, pv.x, rv.x);
        pv.y = fma(beta, pv.y, rv.y);
        sv.x = fma(beta, sv.x, wv.x);
        sv.y = fma(beta, sv.y, wv.y);
        xv.x = fma(alpha, pv.x, xv.x);
        xv.y = fma(alpha, pv.y, xv.y);
        rv.x = fma(-alpha, sv.x, rv.x);
        rv.y = fma(-alpha, sv.y, rv.y);
        x2[q] = xv;
        r2[q] = rv;
        p2[q] = pv;
        s2[q] = sv;
    }
    for (int64_t row = npk * 2 + tid; row < m; row += nth) {
        const double pi = fma(beta, p[row], r[row]);
        const double si = fma(beta, s[row], w[row]);
        p[row] = pi;
        s[row] = si;
        x[row] = fma(alpha, pi, x[row]);
        r[row] = fma(-alpha, si, r[row]);
    }
}

template <int FMT, class VT>
__global__ void __launch_bounds__(kCgThreads, k_cg_min_blocks<FMT>()) k_cg_sr(const CgSrArgs a) {
    __shared__ CgBlockState st;
    __shared__ SrState sr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = (int)a.A.n_rows, ns = (int)a.A.n_slices;
    const int tw = gridDim.x * kCgWarps;
    if (threadIdx.x == 0) {
        st.target = 0;
        st.round = 0;
        st.k = 0;
        st.ok = 1;
        sr.gamma = 0.0;
    }
    __syncthreads();
    int status = FE_ERR_MAXIT;
    bool alive = true;

    // r = b - A x, p = s = 0; b.b
    {
        double bb_part = 0.0;
        for (int sl = blockIdx.x * kCgWarps + warp; sl < ns; sl += tw) {
            const double ax = slice_spmv<FMT, VT, double, double, false>(a.A, sl, lane, a.x);
            const int row = sl * kSlice + lane;
            if (row < m) {
                const double bi = a.b[row];
                a.r[row] = bi - ax;
                a.p[row] = 0.0;
                a.s[row] = 0.0;
                bb_part = fma(bi, bi, bb_part);
            }
        }
        double bb;
        alive = grid_sum1(a, &st, bb_part, bb);
        if (threadIdx.x == 0) st.bb = bb;
        __syncthreads();
    }
    if (alive && st.bb == 0.0) {  // b = 0: the solution is 0
        for (int sl = blockIdx.x * kCgWarps + warp; sl < ns; sl += tw) {
            const int row = sl * kSlice + lane;
            if (row < m) a.x[row] = 0.0;
        }
        if (threadIdx.x == 0) sr.gamma = 0.0;
        status = FE_OK;
    } else if (alive) {
        bool first = true;
        while (true) {
            // S: w = A r, gamma = r.r, delta = w.r
            double g_part = 0.0, d_part = 0.0;
            for (int sl = blockIdx.x * kCgWarps + warp; sl < ns; sl += tw) {
                const double y = slice_spmv<FMT, VT, double, double, false, k_cg_unroll<FMT>()>(a.A, sl, lane, a.r);
                const int row = sl * kSlice + lane;
                if (row < m) {
                    a.w[row] = y;
                    const double ri = a.r[row];
                    g_part = fma(ri, ri, g_part);
                    d_part = fma(y, ri, d_part);
                }
            }
            double gamma, delta;
            if (!(alive = grid_sum2(a, &st, g_part, d_part, gamma, delta))) break;
            // every thread read sr at the top of the previous step; grid_sum2 synchronised the block
            // thread 0 forms the step's scalars (three FP64 divisions once per
            // block instead of in every warp) and the barrier below publishes them
            if (threadIdx.x == 0) {
                if (!first) st.k += 1;
                sr.gamma_prev = first ? 0.0 : sr.gamma;
                sr.gamma = gamma;
                sr.delta = delta;
                double beta = 0.0, curv = delta;
                if (!first) {
                    beta = gamma / sr.gamma_prev;
                    curv = delta - beta * gamma / sr.alpha_prev;
                    if (!(curv > 0.0) || !(curv < INFINITY)) {  // lost its sign: restart the direction
                        beta = 0.0;
                        curv = delta;
                    }
                }
                sr.beta = beta;
                sr.curv = curv;
                sr.alpha = gamma / curv;
            }
            __syncthreads();
            if (sr.gamma <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
            const double beta = sr.beta, curv = sr.curv;
            if (!(curv > 0.0) || !(curv < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            const double alpha = sr.alpha;
            // U
            update_sr(a.x, a.r, a.p, a.s, a.w, m, alpha, beta);
            if (!(alive = grid_barrier(a.ctrl, &st, a.timeout_ns, a.stall_barrier))) break;
            // grid_barrier synchronised the block: nobody still reads sr.alpha_prev
            if (threadIdx.x == 0) sr.alpha_prev = alpha;
            first = false;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = st.k;
        a.ctrl->rr = sr.gamma;
        a.ctrl->bb = st.bb;
    }
}

static size_t cg_sr_workspace_bytes(const fe_matrix &A) {
    const size_t vec = align256((size_t)A.n_slices * kSlice * sizeof(double));
    return 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) + 4 * vec;
}

template <int FMT, class VT> static fe_status launch_cg_sr(const CgSrArgs &args, cudaStream_t s) {
    auto kern = k_cg_sr<FMT, VT>;
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, 0));
    if (per_sm < 1) return FE_ERR_CUDA;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (args.A.n_slices + kCgWarps - 1) / kCgWarps;
    if (blocks > need) blocks = need;
    if (blocks > kCgMaxBlocks) blocks = kCgMaxBlocks;
    if (blocks < 1) blocks = 1;
    void *params[] = {(void *)&args};
    FE_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)blocks), dim3(kCgThreads),
                                            params, 0, s));
    return FE_OK;
}

static fe_status dispatch_cg_sr(const CgSrArgs &args, cudaStream_t s) {
    FE_DISPATCH_FMT_VT(args.A, launch_cg_sr, args, s)
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_cg_sr_workspace(const fe_matrix *A, size_t *h_bytes) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (h_bytes == nullptr) return FE_ERR_ARG;
    *h_bytes = cg_sr_workspace_bytes(*A);
    return FE_OK;
}

fe_status fe_cg_solve_sr(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                         double timeout_s, void *d_work, size_t work_bytes, fe_cg_result *h_result,
                         fe_stream_t stream) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (!d_b || !d_x || !d_work || !h_result || maxit < 0 || !(tol >= 0.0)) return FE_ERR_ARG;
    if (A->n_rows != A->n_cols) return FE_ERR_ARG;
    if (!aligned(d_b, 16) || !aligned(d_x, 16) || !aligned(d_work, 256)) return FE_ERR_ARG;
    if (work_bytes < cg_sr_workspace_bytes(*A)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;

    char *ws = (char *)d_work;
    CgSrArgs args;
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
    args.s = (double *)(v0 + 3 * vec);
    args.tol2 = tol * tol;
    args.maxit = maxit;
    const double tmo = timeout_s > 0.0 ? timeout_s : 2.0;
    args.timeout_ns = (long long)(tmo * 1e9);
    args.stall_barrier = take_stall_barrier();
    args.x0_zero = 0;
    args.x64 = nullptr;

    FE_TRY_CUDA(cudaMemsetAsync(args.ctrl, 0, sizeof(CgCtrl), s));
    st = dispatch_cg_sr(args, s);
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

}  // extern "C"
