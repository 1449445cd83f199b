// fe_cg_resident.cu -- the fused CG (paper Sec. 1: MATVEC, DOT, WAXPY) for
// systems small enough that every warp of the grid owns at most one 32-row
// slice (up to ~38k rows on 152 SMs): the latency-bound case, where a step's
// time is the chain of memory round trips and grid reductions, not the matrix
// stream.
//
// Each warp loads its slice's stored entries (BCRS3 or sliced-ELL, FP64
// values) into registers once, and each lane keeps its row's x, r, p and w in
// registers for the whole solve.  A step is the two-phase textbook step of
// fe_cg.cu (k_cg2):
//   A  gather p_k[j] = beta p_{k-1}[j] + r[j] at the slice's columns (one round
//      of loads from L2), w = A p_k from registers, own row: p_k, x += alpha p
//      in registers, store p_k for the other warps' gathers; reduce p_k.w
//   B  r -= alpha w in registers, store r for the next gathers; reduce r.r
// so a step moves 16 bytes per row to memory plus the gathers, and x goes to
// memory once, at the end.  The operations per row are those of the other
// forms; the dot products' partial sums are per row instead of per 16-byte
// pack, so the bits can differ from fe_cg.cu's kernels in the last place.
// Slots past the register capacity (only for a matrix wider than the 27-point
// stencil) are read from memory every step.
#include "fe_cg_common.cuh"

namespace fe {

template <int FMT> struct ResidentShape;
template <> struct ResidentShape<FE_FMT_BCRS3> { static constexpr int W = 9, T = 3; };
template <> struct ResidentShape<FE_FMT_SELL> { static constexpr int W = 27, T = 1; };

template <int FMT>
__global__ void __launch_bounds__(kCgThreads, 1) k_cg_resident(const CgArgs<double> a) {
    constexpr int W = ResidentShape<FMT>::W, T = ResidentShape<FMT>::T;
    __shared__ CgBlockState st;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = (int)a.A.n_rows;
    const int slice = blockIdx.x * kCgWarps + warp;          // at most one per warp
    const bool has = slice < (int)a.A.n_slices;
    const int row = slice * kSlice + lane;
    const bool live = has && row < m;
    if (threadIdx.x == 0) {
        st.target = 0;
        st.round = 0;
        st.k = 0;
        st.ok = 1;
    }
    // the slice's entries: column (BCRS3: first of three) and values per slot
    int w = 0;
    int64_t base = 0;
    int32_t col[W];
    double val[W][T];
    const double *vals = reinterpret_cast<const double *>(a.A.d_vals);
    if (has) {
        base = a.A.d_slice_ptr[slice];
        w = (int)((a.A.d_slice_ptr[slice + 1] - base) >> 5);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
        col[k] = 0;
#pragma unroll
        for (int t = 0; t < T; ++t) val[k][t] = 0.0;
        if (k < w) {
            col[k] = a.A.d_cols[base + 32 * k + lane];
#pragma unroll
            for (int t = 0; t < T; ++t) val[k][t] = vals[T * base + 32 * T * k + 32 * t + lane];
        }
    }
    __syncthreads();
    // row product of the slice with the operand g(j)
    auto row_product = [&](auto g) {
        double acc = 0.0;
        double xv[W][T];
#pragma unroll
        for (int k = 0; k < W; ++k)
#pragma unroll
            for (int t = 0; t < T; ++t) xv[k][t] = k < w ? g((int64_t)col[k] + t) : 0.0;
#pragma unroll
        for (int k = 0; k < W; ++k)
#pragma unroll
            for (int t = 0; t < T; ++t)
                if (k < w) acc = fma(val[k][t], xv[k][t], acc);
        for (int k = W; k < w; ++k) {           // wider than the register capacity
            const int32_t c = a.A.d_cols[base + 32 * k + lane];
#pragma unroll
            for (int t = 0; t < T; ++t)
                acc = fma(vals[T * base + 32 * T * k + 32 * t + lane], g((int64_t)c + t), acc);
        }
        return acc;
    };

    int status = FE_ERR_MAXIT;
    bool alive = true;
    double xr = 0.0, rr_ = 0.0, pr = 0.0, wr = 0.0;    // own row: x, r, p_{k-1}, w
    // the scalars of the recurrence, the same in every thread (each computes
    // them from the same reduced sums), so no block barrier publishes them
    double rr_cur = 0.0, bb = 0.0, alpha_old = 0.0, beta = 0.0;
    int k = 0;
    {
        const PtrGather<false, double> gx{a.x};
        const double ax = has ? row_product(gx) : 0.0;
        double s0 = 0.0, s1 = 0.0;
        if (live) {
            xr = a.x[row];
            const double bi = a.b[row];
            rr_ = bi - ax;
            pr = rr_;
            a.r[row] = rr_;
            a.p2[row] = rr_;                    // stands for p_{-1}: p_0 = 0 * r + r
            s0 = rr_ * rr_;
            s1 = bi * bi;
        }
        alive = grid_sum2(a, &st, s0, s1, rr_cur, bb);
    }
    if (alive && bb == 0.0) {              // b = 0: the solution is 0
        xr = 0.0;
        rr_cur = 0.0;
        status = FE_OK;
    } else {
        while (alive) {
            if (rr_cur <= a.tol2 * bb) { status = FE_OK; break; }
            if (k >= a.maxit) { status = FE_ERR_MAXIT; break; }
            double *pnew = (k & 1) ? a.p2 : a.p;
            const double *pold = (k & 1) ? a.p : a.p2;
            // A: p_k at the gathered columns, w = A p_k; own row in registers
            const AxpyGather<double> gat{a.r, pold, beta};
            double pw_part = 0.0;
            if (has) {
                const double y = row_product(gat);
                if (live) {
                    const double pk = fma(beta, pr, rr_);
                    xr = fma(alpha_old, pr, xr);
                    pr = pk;
                    wr = y;
                    pnew[row] = pk;
                    pw_part = pk * y;
                }
            }
            double pw, alpha;                // alpha = rr / (p.w), formed once per block
            if (!(alive = grid_sum1_div<1>(a, &st, pw_part, rr_cur, pw, alpha))) break;
            if (!(pw > 0.0) || !(pw < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            // B: r -= alpha w in registers, stored for the next gathers; r.r
            double rr_part = 0.0;
            if (live) {
                rr_ = fma(-alpha, wr, rr_);
                a.r[row] = rr_;
                rr_part = rr_ * rr_;
            }
            double rr_new;                   // beta = r.r / rr, formed once per block
            if (!(alive = grid_sum1_div<2>(a, &st, rr_part, rr_cur, rr_new, beta))) break;
            alpha_old = alpha;
            rr_cur = rr_new;
            k += 1;
            if (rr_new <= a.tol2 * bb) { status = FE_OK; break; }
            if (k >= a.maxit) { status = FE_ERR_MAXIT; break; }
        }
    }
    // the last step's x update (x += alpha_{k-1} p_{k-1}), then x to memory
    if (alive && k > 0 && (status == FE_OK || status == FE_ERR_MAXIT)) xr = fma(alpha_old, pr, xr);
    if (live) a.x[row] = xr;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = k;
        a.ctrl->rr = rr_cur;
        a.ctrl->bb = bb;
    }
}

template <int FMT>
static fe_status launch_resident(const CgArgs<double> &args, cudaStream_t s, bool *taken) {
    auto kern = k_cg_resident<FMT>;
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, 0));
    // 8 slices per block: fewer blocks in each grid reduction (spreading N = 30's
    // 931 slices 7 per block over 133 SMs, less FP64 work per SM, was slower)
    const int64_t blocks = (args.A.n_slices + kCgWarps - 1) / kCgWarps;
    if (per_sm < 1 || blocks > (int64_t)sm_count() * per_sm || blocks > kCgMaxBlocks) {
        *taken = false;                  // the grid would not be co-resident
        return FE_OK;
    }
    void *params[] = {(void *)&args};
    FE_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)blocks), dim3(kCgThreads),
                                            params, 0, s));
    *taken = true;
    return FE_OK;
}

bool resident_cg_fits(const fe_matrix &A) {
    if (A.value_type != FE_VAL_F64 || (A.format != FE_FMT_BCRS3 && A.format != FE_FMT_SELL)) return false;
    const int64_t blocks = (A.n_slices + kCgWarps - 1) / kCgWarps;   // one block of 8 warps per SM
    return blocks <= sm_count();
}

fe_status launch_cg_resident(const CgArgs<double> &args, cudaStream_t s, bool *taken) {
    *taken = false;
    if (!resident_cg_fits(args.A)) return FE_OK;
    if (args.A.format == FE_FMT_BCRS3) return launch_resident<FE_FMT_BCRS3>(args, s, taken);
    return launch_resident<FE_FMT_SELL>(args, s, taken);
}

}  // namespace fe
