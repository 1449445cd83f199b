// fe_cg_mixed.cu -- mixed-precision form of the CG solve (not in the paper;
// it must meet the FP64 path's true-residual test): matrix values stored in FP32 or BF16, the
// Krylov iteration in FP32 with FP32 accumulation, and the residual
// recompute, the refinement update and every global dot product in FP64.
//
// Two modes:
//   FE_MIXED_RELIABLE (default)  one persistent cooperative kernel.  The FP32
//       CG accumulates its correction in an FP32 vector; whenever its residual
//       has dropped by `inner_tol` since the last refinement step (or looks
//       converged), the kernel adds the correction to the FP64 x, recomputes
//       r = b - A64 x with the FP64 matrix, stores it as the FP32 residual and
//       continues with the same search direction ("reliable updates",
//       Sleijpen & van der Vorst 1996).  The Krylov space is never thrown away,
//       so the step count stays close to the FP64 solve's.
//   FE_MIXED_RESTART  a host loop: FP64 residual, FP32 CG from zero to
//       inner_tol, FP64 update; each inner solve starts a new Krylov space.
#include "fe_cg_common.cuh"

namespace fe {

static size_t mixed_workspace_bytes(const fe_matrix &lo) {
    const size_t vec = align256((size_t)lo.n_slices * kSlice * sizeof(float));
    return 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) +
           align256(FE_RESID_WORK_BYTES) + 5 * vec;
}

// Refinement steps in a row without halving the true residual before the
// reliable-update solve gives up (FE_ERR_MAXIT).
constexpr int kMaxStalls = 4;
// FP32 steps after which a refinement step is forced (a plateaued FP32
// residual would otherwise never trigger one).
constexpr int kForceRefineSteps = 256;

struct MixArgs {
    fe_matrix A_lo, A_hi;
    const double *b;
    double *x;                 // FP64 iterate (caller's)
    float *r, *p, *w, *xs;     // FP32 residual, direction, A p, correction since the last update
    double *part;
    CgCtrl *ctrl;
    double tol2, delta2;
    int maxit, max_updates;
    long long timeout_ns;
    long long stall_barrier;
};

// r = b - A_hi x in FP64, stored as FP32 in r (and p when `set_p`); returns
// this thread's partials of r.r and b.b in FP64.
template <int FH>
__device__ __forceinline__ void fp64_residual(const MixArgs &a, int m, int ns, bool set_p,
                                              double &s0, double &s1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tw = gridDim.x * kCgWarps;
    s0 = 0.0;
    s1 = 0.0;
    for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
        const double ax = slice_spmv<FH, double, double, double, false>(a.A_hi, s, lane, a.x);
        const int row = s * kSlice + lane;
        if (row < m) {
            const double bi = a.b[row], ri = bi - ax;
            a.r[row] = (float)ri;
            if (set_p) {
                a.p[row] = (float)ri;
                a.xs[row] = 0.0f;
            }
            s0 = fma(ri, ri, s0);
            s1 = fma(bi, bi, s1);
        }
    }
}

// x += xs, xs = 0 (the FP64 refinement update)
__device__ __forceinline__ void fold_correction(double *x, float *xs, int m) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int npk = m / 4;
    float4 *xs4 = reinterpret_cast<float4 *>(xs);
    double2 *x2 = reinterpret_cast<double2 *>(x);
    for (int q = tid; q < npk; q += nth) {
        const float4 c = xs4[q];
        double2 lo = x2[2 * q], hi = x2[2 * q + 1];
        lo.x += (double)c.x;
        lo.y += (double)c.y;
        hi.x += (double)c.z;
        hi.y += (double)c.w;
        x2[2 * q] = lo;
        x2[2 * q + 1] = hi;
        xs4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int row = npk * 4 + tid; row < m; row += nth) {
        x[row] += (double)xs[row];
        xs[row] = 0.0f;
    }
}

// The inner (low-precision) BCRS3 SpMV was latency-bound with its matrix
// loads issued by the threads.  It streams the matrix through a shared-memory
// ring filled by bulk copies (below); arrays that are not 16-byte aligned take
// the thread-load walk, which puts all nine slots of a 27-point row in flight
// in one trip and the next slice's indices with them (bcrs3_slices_prefetch).

// ------------------------------------------- inner BCRS3 SpMV staged by bulk copies
// Each warp owns kRing stages of shared memory.  Lane 0 streams the column
// indices and values of the warp's slices into them with cp.async.bulk (the
// bytes counted on the stage's mbarrier), kRing slices ahead of the slice the
// warp computes, so the matrix stream stays in flight while the warp gathers
// the operands and multiplies; the warp itself only waits on the gathers.
// A stage: a 16-byte header (the slice's first slot and its width, written by
// lane 0 before its arrive), the 9 x 32 column indices, the 27 x 32 values.
// Slices wider than nine slots are not staged (the header says so) and go
// through slice_spmv_bcrs3 from global memory.
template <class VT> struct MixStage {
    // stages per warp (three BF16 stages measured 3 % slower than two)
    static constexpr int kRing = 2;
    static_assert((kRing & (kRing - 1)) == 0, "the fill count maps to stage and parity by kRing | 2^32");
    static constexpr int kIdx = 16;
    static constexpr int kVal = kIdx + 9 * kSlice * 4;
    static constexpr int kBytes = kVal + 27 * kSlice * (int)sizeof(VT);
    static constexpr size_t kBlockBytes = (size_t)kCgWarps * kRing * kBytes + (size_t)kCgWarps * kRing * 8;
};

__device__ __forceinline__ uint32_t mix_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ long long mix_now() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of a stage's mbarrier; false after 1 s.
__device__ __forceinline__ bool mix_stage_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    long long t0 = 0;
    for (unsigned it = 0; it < (1u << 26); ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (it == 0) t0 = mix_now();
        else if ((it & 255u) == 0 && mix_now() - t0 > 1000000000LL) return false;
    }
    return false;
}

// Lane 0: fill stage `st` of the warp's ring with slice (b, w) (slot offset,
// width); every fill completes the stage's mbarrier phase exactly once.
template <class VT>
__device__ __forceinline__ void mix_stage_fill(const fe_matrix &A, unsigned char *ring, uint32_t bars, int st,
                                               int64_t b, int w, uint64_t policy) {
    unsigned char *dst = ring + (size_t)st * MixStage<VT>::kBytes;
    const uint32_t bar = bars + 8u * (uint32_t)st;
    *reinterpret_cast<int64_t *>(dst) = b;
    *reinterpret_cast<int *>(dst + 8) = w;
    if (w > 0 && w <= 9) {
        const uint32_t ib = (uint32_t)w * kSlice * 4u, vb = (uint32_t)w * 3u * kSlice * (uint32_t)sizeof(VT);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(ib + vb)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
            ::"r"(mix_smem(dst + MixStage<VT>::kIdx)), "l"(A.d_cols + b), "r"(ib), "r"(bar), "l"(policy)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
            ::"r"(mix_smem(dst + MixStage<VT>::kVal)), "l"(reinterpret_cast<const VT *>(A.d_vals) + 3 * b), "r"(vb),
              "r"(bar), "l"(policy)
            : "memory");
    } else {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    }
}

// The warp's grid-stride walk over slices s0, s0 + stride, ... of the inner
// matrix through its ring.  `fills` counts the ring's fills over the kernel's
// life: fill f goes to stage f mod kRing and completes that stage's mbarrier
// phase of parity (f / kRing) mod 2 (kRing a power of two, so both stay right
// when the 32-bit count wraps).  The FMA order is slice_spmv_bcrs3's, so
// results are bitwise the same.  out(s, y, x_row) receives lane's row sum of
// slice s and, for BF16 values, x at lane's row (0 otherwise).  Returns false
// if a stage never completed (after a bounded drain of the fills still in
// flight).
template <class VT, class F>
__device__ __forceinline__ bool bcrs3_slices_staged(const fe_matrix &A, int64_t s0, int64_t stride, int lane,
                                                    const float *x, unsigned char *ring, uint32_t bars,
                                                    uint32_t &fills, F &&out) {
    constexpr int kRing = MixStage<VT>::kRing;
    const int64_t ns = A.n_slices;
    const int64_t n = s0 < ns ? (ns - 1 - s0) / stride + 1 : 0;
    if (n == 0) return true;
    const int64_t *sp = A.d_slice_ptr;
    uint64_t policy = 0;
    int64_t nb = 0;   // lane 0: bounds of the next slice to fill
    int nw = 0;
    if (lane == 0) {
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
        const int64_t q0 = n < kRing ? n : kRing;
        for (int64_t q = 0; q < q0; ++q) {
            const int64_t s = s0 + q * stride;
            const int64_t b = sp[s];
            mix_stage_fill<VT>(A, ring, bars, (int)((fills + q) % kRing), b, (int)((sp[s + 1] - b) >> 5),
                               policy);
        }
        if (n > kRing) {
            const int64_t s = s0 + kRing * stride;
            nb = sp[s];
            nw = (int)((sp[s + 1] - nb) >> 5);
        }
    }
    bool ok = true;
    int64_t q = 0;
    for (; q < n; ++q) {
        const uint32_t f = fills + (uint32_t)q;
        const int st = (int)(f % kRing);
        if (!__all_sync(0xffffffffu, mix_stage_wait(bars + 8u * (uint32_t)st, (f / kRing) & 1u))) {
            ok = false;
            break;
        }
        const unsigned char *stage = ring + (size_t)st * MixStage<VT>::kBytes;
        const int w = *reinterpret_cast<const int *>(stage + 8);
        const int64_t s = s0 + q * stride;
        // BF16 values: x at lane's row goes out with the gathers (measured 1-3 %
        // less time per step); FP32 values: out() loads it (the early load
        // measured 5 % slower there)
        float xr = 0.0f;
        if constexpr (sizeof(VT) == 2) {
            const int64_t row = s * kSlice + lane;
            xr = row < A.n_rows ? x[row] : 0.0f;
        }
        float acc = 0.0f;
        if (w == 9) {
            const int32_t *si = reinterpret_cast<const int32_t *>(stage + MixStage<VT>::kIdx) + lane;
            const VT *sv = reinterpret_cast<const VT *>(stage + MixStage<VT>::kVal) + lane;
            float xx[9][3];
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                const int64_t j = si[32 * u];
#pragma unroll
                for (int t = 0; t < 3; ++t) xx[u][t] = x[j + t];
            }
#pragma unroll
            for (int u = 0; u < 9; ++u)
#pragma unroll
                for (int t = 0; t < 3; ++t) acc = fmaf(to_acc<float>(sv[96 * u + 32 * t]), xx[u][t], acc);
        } else if (w > 0 && w < 9) {
            const int32_t *si = reinterpret_cast<const int32_t *>(stage + MixStage<VT>::kIdx) + lane;
            const VT *sv = reinterpret_cast<const VT *>(stage + MixStage<VT>::kVal) + lane;
            for (int k = 0; k < w; ++k) {
                const int64_t j = si[32 * k];
#pragma unroll
                for (int t = 0; t < 3; ++t) acc = fmaf(to_acc<float>(sv[96 * k + 32 * t]), x[j + t], acc);
            }
        } else if (w > 9) {
            acc = slice_spmv_bcrs3<VT, float, float, 9>(A, s, lane, PtrGather<false, float>{x});
        }
        __syncwarp();
        // every lane has consumed the stage: lane 0 refills it kRing slices ahead
        if (lane == 0 && q + kRing < n) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mix_stage_fill<VT>(A, ring, bars, st, nb, nw, policy);
            if (q + kRing + 1 < n) {
                const int64_t sn = s0 + (q + kRing + 1) * stride;
                nb = sp[sn];
                nw = (int)((sp[sn + 1] - nb) >> 5);
            }
        }
        out(s, acc, xr);
    }
    if (!ok) {
        // drain: wait (bounded) for every fill issued but not consumed
        const int64_t issued = n < q + kRing ? n : q + kRing;
        for (int64_t d = q; d < issued; ++d) {
            const uint32_t f = fills + (uint32_t)d;
            mix_stage_wait(bars + 8u * (f % kRing), (f / kRing) & 1u);
        }
    }
    fills += (uint32_t)n;
    return ok;
}

// Blocks per SM: four for BF16 BCRS3 values (64 registers; the staged form's
// 46.5 KB ring per block fits four times; measured 6 % less time per inner
// step than three), three for FP32 BCRS3 values and the CSR forms (80
// registers; the FP32 ring's 74 KB per block allows no more).  The staged and
// thread-load forms of one value type take the same block count, hence the
// same grid, the same reduction order and bitwise the same solve.
template <int FL, class VL, int FH>
constexpr int mix_min_blocks() {
    if (FL == FE_FMT_BCRS3 && sizeof(VL) == 2) return 4;
    return (FL == FE_FMT_CSR || FH == FE_FMT_CSR || FL == FE_FMT_BCRS3) ? 3 : kCgBlocksPerSm;
}

template <int FL, class VL, int FH, bool STAGED = false>
__global__ void __launch_bounds__(kCgThreads, mix_min_blocks<FL, VL, FH>())
k_cg_reliable(const MixArgs a) {
    __shared__ CgBlockState st;
    __shared__ double s_rr_max;
    __shared__ double s_rr_true;   // last FP64 true residual (reported)
    __shared__ int s_updates;
    __shared__ int s_stalls;       // refinement steps in a row that did not halve the residual
    __shared__ int s_last_refine;  // step count at the last refinement
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = (int)a.A_lo.n_rows, ns = (int)a.A_lo.n_slices;
    const int tw = gridDim.x * kCgWarps;
    unsigned char *ring = nullptr;   // STAGED: this warp's stages and mbarriers
    uint32_t bars = 0, fills = 0;
    if constexpr (STAGED) {
        extern __shared__ __align__(128) unsigned char mix_dyn[];
        constexpr int kRing = MixStage<VL>::kRing;
        ring = mix_dyn + (size_t)warp * kRing * MixStage<VL>::kBytes;
        bars = mix_smem(mix_dyn + (size_t)kCgWarps * kRing * MixStage<VL>::kBytes) + 8u * kRing * (uint32_t)warp;
        if (lane == 0) {
            for (int i = 0; i < kRing; ++i)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bars + 8u * i), "r"(1));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if (threadIdx.x == 0) {
        st.target = 0;
        st.round = 0;
        st.k = 0;
        st.ok = 1;
        s_updates = 0;
        s_stalls = 0;
        s_last_refine = 0;
    }
    __syncthreads();
    int status = FE_ERR_MAXIT;
    bool alive = true;
    double s0, s1, rr_true, bb;
    fp64_residual<FH>(a, m, ns, true, s0, s1);
    alive = grid_sum2(a, &st, s0, s1, rr_true, bb);
    if (threadIdx.x == 0) {
        st.rr = rr_true;
        st.bb = bb;
        s_rr_max = rr_true;
        s_rr_true = rr_true;
    }
    __syncthreads();
    if (alive && bb == 0.0) {  // b = 0: the solution is 0
        const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
        for (int row = tid; row < m; row += nth) a.x[row] = 0.0;
        if (threadIdx.x == 0) s_rr_true = 0.0;
        status = FE_OK;
    } else if (alive && rr_true <= a.tol2 * bb) {
        status = FE_OK;
    } else {
        while (alive) {
            // A: w = A_lo p (FP32), p.w
            float pw_part = 0.0f;
            auto out = [&](int64_t s, float y, float p_row) {
                const int row = (int)s * kSlice + lane;
                if (row < m) {
                    a.w[row] = y;
                    pw_part = fmaf(sizeof(VL) == 2 ? p_row : a.p[row], y, pw_part);
                }
            };
            if constexpr (STAGED) {
                const bool ok = bcrs3_slices_staged<VL>(a.A_lo, blockIdx.x * kCgWarps + warp, tw, lane, a.p,
                                                        ring, bars, fills, out);
                if (!ok && lane == 0) atomicExch(&a.ctrl->abort, 1);  // the other blocks leave at their barrier
                if (__syncthreads_or(!ok)) { alive = false; break; }
            } else if constexpr (FL == FE_FMT_BCRS3) {
                bcrs3_slices_prefetch<VL, float, float>(a.A_lo, blockIdx.x * kCgWarps + warp, tw, lane,
                                                        PtrGather<false, float>{a.p}, out);
            } else {
                for (int s = blockIdx.x * kCgWarps + warp; s < ns; s += tw) {
                    const int row = s * kSlice + lane;
                    const float pr = row < m ? a.p[row] : 0.0f;
                    out(s, slice_spmv<FL, VL, float, float, false>(a.A_lo, s, lane, a.p), pr);
                }
            }
            double pw, alpha;                // alpha = rr / (p.w), formed once per block
            if (!(alive = grid_sum1_div<1>(a, &st, (double)pw_part, st.rr, pw, alpha))) break;
            if (!(pw > 0.0) || !(pw < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            // B: xs += alpha p, r -= alpha w, r.r
            const float rr_part = update_xr<float>(a.xs, a.r, a.p, a.w, m, (float)alpha);
            double rr_new;
            if (!(alive = grid_sum1(a, &st, (double)rr_part, rr_new))) break;
            __syncthreads();
            if (threadIdx.x == 0) st.k += 1;
            __syncthreads();
            const bool refine = rr_new <= a.delta2 * s_rr_max || rr_new <= a.tol2 * st.bb ||
                                st.k >= a.maxit || st.k - s_last_refine >= kForceRefineSteps;
            if (refine) {
                // x += xs in FP64, then r = b - A64 x in FP64 (stored as the FP32 residual)
                fold_correction(a.x, a.xs, m);
                if (!(alive = grid_barrier(a.ctrl, &st, a.timeout_ns, a.stall_barrier))) break;
                fp64_residual<FH>(a, m, ns, false, s0, s1);
                if (!(alive = grid_sum1(a, &st, s0, rr_true))) break;
                __syncthreads();
                if (threadIdx.x == 0) {
                    s_updates += 1;
                    s_last_refine = st.k;
                    // the true residual must keep falling; if the low-precision
                    // operator is too far from A64 (delta * cond(A) ~ 1) it stalls
                    s_stalls = (rr_true > 0.25 * s_rr_true) ? s_stalls + 1 : 0;
                    s_rr_max = rr_true;
                    s_rr_true = rr_true;
                }
                __syncthreads();
                rr_new = rr_true;
                if (rr_true <= a.tol2 * st.bb) { status = FE_OK; break; }
                if (st.k >= a.maxit || s_updates >= a.max_updates || s_stalls >= kMaxStalls) {
                    status = FE_ERR_MAXIT;
                    break;
                }
            }
            const double beta = rr_new / st.rr;
            __syncthreads();
            if (threadIdx.x == 0) st.rr = rr_new;
            __syncthreads();
            // C: p = r + beta p
            update_p<float>(a.p, a.r, m, (float)beta);
            if (!(alive = grid_barrier(a.ctrl, &st, a.timeout_ns, a.stall_barrier))) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = st.k;
        a.ctrl->pad = s_updates;
        a.ctrl->rr = s_rr_true;
        a.ctrl->bb = st.bb;
    }
}

template <int FL, class VL, int FH, bool STAGED = false>
static fe_status launch_reliable(const MixArgs &args, cudaStream_t s) {
    auto kern = k_cg_reliable<FL, VL, FH, STAGED>;
    const size_t dyn = STAGED ? MixStage<VL>::kBlockBytes : 0;
    if (STAGED) FE_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, dyn));
    if (per_sm < 1) return FE_ERR_CUDA;
    int64_t blocks = (int64_t)sm_count() * per_sm;
    const int64_t need = (args.A_lo.n_slices + kCgWarps - 1) / kCgWarps;
    if (blocks > need) blocks = need;
    if (blocks > kCgMaxBlocks) blocks = kCgMaxBlocks;
    if (blocks < 1) blocks = 1;
    void *params[] = {(void *)&args};
    FE_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)blocks), dim3(kCgThreads),
                                            params, dyn, s));
    return FE_OK;
}

template <int FL, class VL, bool STAGED = false>
static fe_status dispatch_reliable_hi(const MixArgs &a, cudaStream_t s) {
    switch (a.A_hi.format) {
        case FE_FMT_CSR: return launch_reliable<FL, VL, FE_FMT_CSR, STAGED>(a, s);
        case FE_FMT_SELL: return launch_reliable<FL, VL, FE_FMT_SELL, STAGED>(a, s);
        case FE_FMT_BCRS3: return launch_reliable<FL, VL, FE_FMT_BCRS3, STAGED>(a, s);
        default: return FE_ERR_ARG;
    }
}

// BCRS3 inner matrices stream through the bulk-copy ring when both arrays
// start on a 16-byte boundary (every slice's block of indices and values then
// does too: a slice starts at a multiple of 32 slots).
template <class VL>
static fe_status dispatch_reliable_bcrs3(const MixArgs &a, cudaStream_t s) {
    if (aligned(a.A_lo.d_cols, 16) && aligned(a.A_lo.d_vals, 16))
        return dispatch_reliable_hi<FE_FMT_BCRS3, VL, true>(a, s);
    return dispatch_reliable_hi<FE_FMT_BCRS3, VL>(a, s);
}

static fe_status dispatch_reliable(const MixArgs &a, cudaStream_t s) {
    switch (a.A_lo.format * 3 + a.A_lo.value_type) {
        case FE_FMT_CSR * 3 + FE_VAL_F32: return dispatch_reliable_hi<FE_FMT_CSR, float>(a, s);
        case FE_FMT_CSR * 3 + FE_VAL_BF16: return dispatch_reliable_hi<FE_FMT_CSR, __nv_bfloat16>(a, s);
        case FE_FMT_SELL * 3 + FE_VAL_F32: return dispatch_reliable_hi<FE_FMT_SELL, float>(a, s);
        case FE_FMT_SELL * 3 + FE_VAL_BF16: return dispatch_reliable_hi<FE_FMT_SELL, __nv_bfloat16>(a, s);
        case FE_FMT_BCRS3 * 3 + FE_VAL_F32: return dispatch_reliable_bcrs3<float>(a, s);
        case FE_FMT_BCRS3 * 3 + FE_VAL_BF16: return dispatch_reliable_bcrs3<__nv_bfloat16>(a, s);
        default: return FE_ERR_ARG;  // FP64 inner values: use fe_cg_solve
    }
}

static fe_status solve_mixed_reliable(const fe_matrix *A64, const fe_matrix *A_lo, const double *d_b,
                                      double *d_x, double tol, int max_outer, double inner_tol,
                                      int max_inner, double timeout_s, void *d_work,
                                      fe_mixed_result *h_result, cudaStream_t s) {
    char *ws = (char *)d_work;
    MixArgs a;
    a.A_lo = *A_lo;
    a.A_hi = *A64;
    a.b = d_b;
    a.x = d_x;
    a.ctrl = (CgCtrl *)ws;
    a.part = (double *)(ws + 256);
    char *q = ws + 256 + align256(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) +
              align256(FE_RESID_WORK_BYTES);
    const size_t vec = align256((size_t)A_lo->n_slices * kSlice * sizeof(float));
    a.r = (float *)q;
    a.p = (float *)(q + vec);
    a.w = (float *)(q + 2 * vec);
    a.xs = (float *)(q + 3 * vec);
    a.tol2 = tol * tol;
    a.delta2 = inner_tol * inner_tol;
    a.maxit = max_inner;
    a.max_updates = max_outer;
    a.timeout_ns = (long long)((timeout_s > 0.0 ? timeout_s : 2.0) * 1e9);
    a.stall_barrier = -1;
    FE_TRY_CUDA(cudaMemsetAsync(a.ctrl, 0, sizeof(CgCtrl), s));
    fe_status st = dispatch_reliable(a, s);
    if (st != FE_OK) return st;
    CgCtrl c;
    FE_TRY_CUDA(cudaMemcpyAsync(&c, a.ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    h_result->status = c.status;
    h_result->outer_iterations = c.pad;
    h_result->inner_iterations = c.iterations;
    h_result->bnorm = sqrt(c.bb);
    h_result->relres = c.bb > 0.0 ? sqrt(c.rr / c.bb) : 0.0;
    return (fe_status)c.status;
}


// Restarted refinement: host loop of FP64 residual -> FP32 CG from zero ->
// FP64 update.  Arguments already checked by the caller.
static fe_status solve_mixed_restart(const fe_matrix *A64, const fe_matrix *A_lo, const double *d_b,
                                     double *d_x, double tol, int max_outer, double inner_tol,
                                     int max_inner, double timeout_s, void *d_work,
                                     fe_mixed_result *h_result, cudaStream_t s) {
    fe_status st = FE_OK;

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
        st = launch_cg_f32(in, s);
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


}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_cg_mixed_workspace(const fe_matrix *A_lo, size_t *h_bytes) {
    fe_status st = check_matrix(A_lo);
    if (st != FE_OK) return st;
    if (h_bytes == nullptr) return FE_ERR_ARG;
    *h_bytes = mixed_workspace_bytes(*A_lo);
    return FE_OK;
}

fe_status fe_cg_solve_mixed(const fe_matrix *A64, const fe_matrix *A_lo, const double *d_b,
                            double *d_x, double tol, int mode, int max_outer, double inner_tol,
                            int max_inner, double timeout_s, void *d_work, size_t work_bytes,
                            fe_mixed_result *h_result, fe_stream_t stream) {
    fe_status st = check_matrix(A64);
    if (st != FE_OK) return st;
    st = check_matrix(A_lo);
    if (st != FE_OK) return st;
    if (A64->value_type != FE_VAL_F64 || A64->n_rows != A64->n_cols ||
        A_lo->n_rows != A64->n_rows || A_lo->n_cols != A64->n_cols)
        return FE_ERR_ARG;
    if (mode != FE_MIXED_RELIABLE && mode != FE_MIXED_RESTART) return FE_ERR_ARG;
    if (mode == FE_MIXED_RELIABLE && A_lo->value_type == FE_VAL_F64) return FE_ERR_ARG;
    if (!d_b || !d_x || !d_work || !h_result || max_outer < 0 || max_inner < 0 || !(tol >= 0.0) ||
        !(inner_tol > 0.0 && inner_tol < 1.0))
        return FE_ERR_ARG;
    if (!aligned(d_b, 16) || !aligned(d_x, 16) || !aligned(d_work, 256)) return FE_ERR_ARG;
    if (work_bytes < mixed_workspace_bytes(*A_lo)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == FE_MIXED_RELIABLE)
        return solve_mixed_reliable(A64, A_lo, d_b, d_x, tol, max_outer, inner_tol, max_inner,
                                    timeout_s, d_work, h_result, s);
    return solve_mixed_restart(A64, A_lo, d_b, d_x, tol, max_outer, inner_tol, max_inner, timeout_s,
                               d_work, h_result, s);
}

}  // extern "C"
