// fe_cg.cu -- unpreconditioned CG (paper Sec. 1: MATVEC + DOT + WAXPY) as
// one persistent cooperative kernel per solve, and the true-residual check.
//
// Each CG step is three phases separated by grid barriers:
//   A  w = A p over the block's slices, p.w accumulated in the SpMV epilogue
//   B  r -= alpha w, r.r accumulated in the same pass
//   C  x += alpha p, p = r + beta p (x is updated where p is read anyway; the
//      last step's x update is applied after the loop)
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
#include "fe_cg_common.cuh"

namespace fe {

template <int FMT, class VT, class XT>
__global__ void __launch_bounds__(kCgThreads, k_cg_min_blocks<FMT>()) k_cg(const CgArgs<XT> a) {
    __shared__ CgBlockState st;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    bool has_pending = false;   // block-uniform
    XT pending = XT(0);

    // r = b - A x, p = r; r.r and b.b
    {
        XT s0 = XT(0), s1 = XT(0);
        for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
            XT ax = XT(0);
            if (!a.x0_zero) ax = slice_spmv<FMT, VT, XT, XT, false>(a.A, s, lane, a.x);
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
                const XT y = slice_spmv<FMT, VT, XT, XT, false, k_cg_unroll<FMT>()>(a.A, s, lane, a.p);
                const int row = s * kSlice + lane;
                if (row < m) {
                    a.w[row] = y;
                    pw_part = fma(a.p[row], y, pw_part);
                }
            }
            double pw, alpha_d;              // alpha = rr / (p.w), formed once per block
            if (!(alive = grid_sum1_div<1>(a, &st, (double)pw_part, st.rr, pw, alpha_d))) break;
            if (!(pw > 0.0) || !(pw < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            // B: r -= alpha w, r.r (x += alpha p is applied in C, where p is read anyway)
            const XT alpha = (XT)alpha_d;
            const XT rr_part = update_r<XT>(a.r, a.w, m, alpha);
            double rr_new, beta;             // beta = r.r / rr, formed once per block
            if (!(alive = grid_sum1_div<2>(a, &st, (double)rr_part, st.rr, rr_new, beta))) break;
            __syncthreads();                 // every thread has read st.rr
            if (threadIdx.x == 0) {
                st.rr = rr_new;
                st.k += 1;
            }
            __syncthreads();
            if (rr_new <= a.tol2 * st.bb || st.k >= a.maxit) {
                status = rr_new <= a.tol2 * st.bb ? FE_OK : FE_ERR_MAXIT;
                pending = alpha;             // the last x update is still to be applied
                has_pending = true;
                break;
            }
            // C: x += alpha p, p = r + beta p
            update_xp<XT>(a.x, a.p, a.r, m, alpha, (XT)beta);
            if (!(alive = grid_barrier(a.ctrl, &st, a.timeout_ns, a.stall_barrier))) break;
        }
    }
    // last x update (row by row; no barrier needed: the fold below uses the
    // same rows per thread), then the refinement step of the mixed-precision
    // form: x64 += x
    if (alive && (status == FE_OK || status == FE_ERR_MAXIT) && (has_pending || a.x64 != nullptr)) {
        const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
        for (int row = tid; row < m; row += nth) {
            XT xi = a.x[row];
            if (has_pending) {
                xi = fma(pending, a.p[row], xi);
                a.x[row] = xi;
            }
            if (a.x64 != nullptr) a.x64[row] += (double)xi;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = st.k;
        a.ctrl->rr = st.rr;
        a.ctrl->bb = st.bb;
    }
}

// Two-phase form of the same iteration, for meshes small enough that the
// grid barriers, not the matrix stream, set the step time.  Phase C of k_cg
// (x += alpha p, p = r + beta p) moves into the next step's SpMV: every
// gathered operand value is formed where it is read, p_k[j] = beta p_{k-1}[j]
// + r[j] (one FMA, the same rounding for every reader), the warp owning row i
// also stores p_k[i] and applies x_i += alpha_{k-1} p_{k-1}[i].  p is double-
// buffered (p_k goes to pbuf[k & 1] while other warps still gather p_{k-1}
// from the other buffer), so a step is
//   A  w = A p_k (operand formed on the fly), p_k.w; x and p for own rows
//   B  r -= alpha w, r.r
// with two grid reductions and no third barrier.  Every value is computed by
// the same operations in the same order as in k_cg, so both forms give
// identical bits; this one reads r and p_{k-1} at each gathered column and
// does one more FMA there, which costs more than a barrier once the FP64
// pipe, not latency, bounds the step.
template <int FMT, class VT>
__global__ void __launch_bounds__(kCgThreads, k_cg_min_blocks<FMT>()) k_cg2(const CgArgs<double> a) {
    __shared__ CgBlockState st;
    __shared__ double coef[2];           // alpha of the last step, beta
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = (int)a.A.n_rows, ns = (int)a.A.n_slices;
    const int tw = gridDim.x * kCgWarps;
    if (threadIdx.x == 0) {
        st.target = 0;
        st.round = 0;
        st.k = 0;
        st.ok = 1;
        coef[0] = coef[1] = 0.0;
    }
    __syncthreads();
    int status = FE_ERR_MAXIT;
    bool alive = true;
    // r = b - A x; pbuf[1] = r stands for p_{-1}, so that step 0 forms
    // p_0 = 0 * r + r = r and applies x += 0 * r
    {
        double s0 = 0.0, s1 = 0.0;
        for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
            double ax = 0.0;
            if (!a.x0_zero) ax = slice_spmv<FMT, VT, double, double, false>(a.A, s, lane, a.x);
            const int row = s * kSlice + lane;
            if (row < m) {
                const double bi = a.b[row];
                const double ri = bi - ax;
                if (a.x0_zero) a.x[row] = 0.0;
                a.r[row] = ri;
                a.p2[row] = ri;
                s0 = fma(ri, ri, s0);
                s1 = fma(bi, bi, s1);
            }
        }
        double rr0, bb0;
        alive = grid_sum2(a, &st, s0, s1, rr0, bb0);
        if (threadIdx.x == 0) {
            st.rr = rr0;
            st.bb = bb0;
        }
        __syncthreads();
    }
    if (alive && st.bb == 0.0) {  // b = 0: the solution is 0
        for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
            const int row = s * kSlice + lane;
            if (row < m) a.x[row] = 0.0;
        }
        if (threadIdx.x == 0) st.rr = 0.0;
        status = FE_OK;
    } else {
        while (alive) {
            if (st.rr <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
            const int k = st.k;
            double *pnew = (k & 1) ? a.p2 : a.p;
            const double *pold = (k & 1) ? a.p : a.p2;
            const double beta = coef[1], alpha_old = coef[0];
            // A: p_k = r + beta p_{k-1} formed at every gathered column, w = A p_k, p_k.w;
            //    own rows: store p_k, x += alpha_{k-1} p_{k-1}
            const AxpyGather<double> gat{a.r, pold, beta};
            double pw_part = 0.0;
            for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
                const double y = slice_spmv_g<FMT, VT, double, double>(a.A, s, lane, gat);
                const int row = s * kSlice + lane;
                if (row < m) {
                    const double po = pold[row];
                    const double pk = fma(beta, po, a.r[row]);
                    a.x[row] = fma(alpha_old, po, a.x[row]);
                    pnew[row] = pk;
                    a.w[row] = y;
                    pw_part = fma(pk, y, pw_part);
                }
            }
            double pw, alpha;                // alpha = rr / (p.w), formed once per block
            if (!(alive = grid_sum1_div<1>(a, &st, pw_part, st.rr, pw, alpha))) break;
            if (!(pw > 0.0) || !(pw < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            // B: r -= alpha w, r.r
            const double rr_part = update_r<double>(a.r, a.w, m, alpha);
            double rr_new;
            if (!(alive = grid_sum1(a, &st, rr_part, rr_new))) break;
            __syncthreads();                 // every thread has read st.rr and coef
            if (threadIdx.x == 0) {
                coef[0] = alpha;
                coef[1] = rr_new / st.rr;
                st.rr = rr_new;
                st.k += 1;
            }
            __syncthreads();
            if (rr_new <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
        }
    }
    // the last step's x update: x += alpha_{k-1} p_{k-1}, p_{k-1} in pbuf[(k-1) & 1]
    if (alive && st.k > 0 && (status == FE_OK || status == FE_ERR_MAXIT)) {
        const double *plast = ((st.k - 1) & 1) ? a.p2 : a.p;
        const double al = coef[0];
        const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
        for (int row = tid; row < m; row += nth) a.x[row] = fma(al, plast[row], a.x[row]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = st.k;
        a.ctrl->rr = st.rr;
        a.ctrl->bb = st.bb;
    }
}

// Workspace: control block, reduction partials, then r, p, w and the second
// p buffer of the two-phase form.
static size_t cg_workspace_bytes(const fe_matrix &A) {
    const size_t vec = align256((size_t)A.n_slices * kSlice * sizeof(double));
    return 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) + 4 * vec;
}

// FE_CG_AUTO: the matrix-resident kernel when A qualifies (FP64 BCRS3 or
// sliced-ELL values, at most one slice per warp of one block per SM), else the
// two-phase form while the whole grid holds at most one slice per warp (every
// warp's SpMV is one pass of its slice, so the step time is the barriers' and
// reductions' latency, not the FP64 pipe's), else the three-phase form.
static int cg_pick_form(const fe_matrix &A, int form) {
    if (form != FE_CG_AUTO) return form;
    if (resident_cg_fits(A)) return FE_CG_RESIDENT;
    const int blocks_per_sm = A.format == FE_FMT_BCRS3 ? k_cg_min_blocks<FE_FMT_BCRS3>() : kCgBlocksPerSm;
    const int64_t warps = (int64_t)sm_count() * blocks_per_sm * kCgWarps;
    return A.n_slices <= warps ? FE_CG_TWO_PHASE : FE_CG_THREE_PHASE;
}

template <int FMT, class VT, class XT>
static fe_status launch_cg(const CgArgs<XT> &args, cudaStream_t s) {
    auto kern = k_cg<FMT, VT, XT>;
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

template <int FMT, class VT> static fe_status launch_cg64(const CgArgs<double> &a, cudaStream_t s) {
    return launch_cg<FMT, VT, double>(a, s);
}
template <int FMT, class VT> static fe_status launch_cg2(const CgArgs<double> &args, cudaStream_t s) {
    auto kern = k_cg2<FMT, VT>;
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
static fe_status dispatch_cg2(const CgArgs<double> &args, cudaStream_t s) {
    FE_DISPATCH_FMT_VT(args.A, launch_cg2, args, s)
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

fe_status launch_cg_f32(const CgArgs<float> &args, cudaStream_t s) { return dispatch_cg(args, s); }

static thread_local long long g_stall_barrier = -1;

long long take_stall_barrier() {
    const long long v = g_stall_barrier;
    g_stall_barrier = -1;
    return v;
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

fe_status fe_cg_solve_form(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                           double timeout_s, int form, void *d_work, size_t work_bytes,
                           fe_cg_result *h_result, fe_stream_t stream) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (!d_b || !d_x || !d_work || !h_result || maxit < 0 || !(tol >= 0.0)) return FE_ERR_ARG;
    if (form != FE_CG_AUTO && form != FE_CG_THREE_PHASE && form != FE_CG_TWO_PHASE &&
        form != FE_CG_RESIDENT)
        return FE_ERR_ARG;
    if (form == FE_CG_RESIDENT && !resident_cg_fits(*A)) return FE_ERR_ARG;
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
    args.p2 = (double *)(v0 + 3 * vec);
    args.tol2 = tol * tol;
    args.maxit = maxit;
    const double tmo = timeout_s > 0.0 ? timeout_s : 2.0;
    args.timeout_ns = (long long)(tmo * 1e9);
    args.stall_barrier = take_stall_barrier();
    args.x0_zero = 0;
    args.x64 = nullptr;

    FE_TRY_CUDA(cudaMemsetAsync(args.ctrl, 0, sizeof(CgCtrl), s));
    const int pick = cg_pick_form(*A, form);
    bool taken = false;
    if (pick == FE_CG_RESIDENT) {
        st = launch_cg_resident(args, s, &taken);
        if (st != FE_OK) return st;
        if (!taken && form == FE_CG_RESIDENT) return FE_ERR_ARG;
    }
    if (!taken) st = (pick == FE_CG_THREE_PHASE) ? dispatch_cg(args, s) : dispatch_cg2(args, s);
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

fe_status fe_cg_solve(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                      double timeout_s, void *d_work, size_t work_bytes, fe_cg_result *h_result,
                      fe_stream_t stream) {
    return fe_cg_solve_form(A, d_b, d_x, tol, maxit, timeout_s, FE_CG_AUTO, d_work, work_bytes,
                            h_result, stream);
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

// ---------------------------------------------------------------- solve without allocation
//
// fe_cg_solve_noalloc serves callers that cannot allocate device memory when
// they solve: code inside a latency-critical loop, where cudaMalloc's implicit
// device-wide synchronisation is not acceptable, or a plugin whose host
// framework owns every device buffer and forbids driver allocations.  They
// still pass A, b and x; the solver's own scratch (barrier/result block,
// reduction partials and the r, p, w vectors) lives in the file-scope array
// below, which every GPU that loads this library holds until the process
// exits.  Host code cannot use the array's name as a device address, so every
// call looks the address up with cudaGetSymbolAddress on the current device.
// The lookup is a host-side query (no allocation, nothing enqueued); doing it
// per call instead of caching it keeps the address valid after a
// cudaDeviceReset, which reloads the module and moves the array.

namespace fe {

constexpr size_t kNoallocVecBytes = ((size_t)FE_NOALLOC_MAX_ROWS * sizeof(double) + 255) & ~(size_t)255;
constexpr size_t kNoallocBytes =
    256 + ((2 * 2 * (size_t)kCgMaxBlocks * sizeof(double) + 255) & ~(size_t)255) + 4 * kNoallocVecBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch on the current device.
static fe_status noalloc_scratch(void **out) {
    void *p = nullptr;
    FE_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = p;
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
