// fe_common.cuh -- shared device/host helpers of libfe (GB300, sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fe.h"

namespace fe {

constexpr int kSlice = FE_SLICE_ROWS;  // rows per slice = one warp

// ---------------------------------------------------------------- host status

void set_cuda_error(cudaError_t e);

#define FE_TRY_CUDA(expr)                              \
    do {                                               \
        cudaError_t fe_e_ = (expr);                    \
        if (fe_e_ != cudaSuccess) {                    \
            ::fe::set_cuda_error(fe_e_);               \
            return FE_ERR_CUDA;                        \
        }                                              \
    } while (0)

#define FE_TRY_LAUNCH() FE_TRY_CUDA(cudaGetLastError())

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Validates a matrix descriptor; returns FE_OK or FE_ERR_ARG / FE_ERR_OVERFLOW.
fe_status check_matrix(const fe_matrix *A);

// Number of SMs of the current device (cached per device).
int sm_count();

// Weight-gradient partials part[split][a][b][t] summed in split order into
// dW[ci][t][co] (a = co and b = ci when a_is_co, else the reverse); fe_nn.cu.
fe_status launch_corr_reduce(const float *part, int n_split, int ca, int cb, int a_is_co, float *dw,
                             cudaStream_t s);

// ---------------------------------------------------------------- device loads

// Matrix streams are read once per pass and are far larger than L2: load them
// with the streaming (evict-first) hint so the vectors stay resident in L2.
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ __nv_bfloat16 ld_stream(const __nv_bfloat16 *p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_bfloat16(u);
}

template <class AT> __device__ __forceinline__ AT to_acc(double v) { return (AT)v; }
template <class AT> __device__ __forceinline__ AT to_acc(float v) { return (AT)v; }
template <class AT> __device__ __forceinline__ AT to_acc(__nv_bfloat16 v) {
    return (AT)__bfloat162float(v);
}

// Gathered vector loads.  `kReadOnly` selects the non-coherent path, valid
// only when the vector is not written during the kernel.
template <bool kReadOnly, class T> __device__ __forceinline__ T ld_vec(const T *p) {
    if constexpr (kReadOnly) return __ldg(p);
    else return *p;
}

// Sum over the warp with an xor butterfly: addition is commutative, so every
// lane ends with the same bits.
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------- slice SpMV

// Operand gathers of the slice SpMV: x[j] from a stored vector, or an operand
// formed on the fly from two vectors (the fused CG step's p = r + beta p_old,
// computed where it is gathered, so that no pass stores p before the SpMV).
template <bool kReadOnly, class XT> struct PtrGather {
    const XT *x;
    __device__ __forceinline__ XT operator()(int64_t j) const { return ld_vec<kReadOnly>(x + j); }
};
template <class XT> struct AxpyGather {   // beta * pold[j] + r[j], one rounding (FMA)
    const XT *r, *pold;
    XT beta;
    __device__ __forceinline__ XT operator()(int64_t j) const { return fma(beta, pold[j], r[j]); }
};

// One warp computes the 32 rows of slice s; returns lane's row sum (0 for
// rows past the end).  XT: vector type, AT: accumulation type.
template <class VT, class XT, class AT, class G>
__device__ __forceinline__ AT slice_spmv_sell(const fe_matrix &A, int64_t s, int lane, const G &x) {
    const int64_t b = A.d_slice_ptr[s];
    const int w = (int)((A.d_slice_ptr[s + 1] - b) >> 5);
    const int32_t *c = A.d_cols + b + lane;
    const VT *v = reinterpret_cast<const VT *>(A.d_vals) + b + lane;
    AT acc = AT(0);
    int k = 0;
    constexpr int U = 9;
    for (; k + U <= w; k += U) {
        int32_t cc[U];
        VT vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = ld_stream(c + 32 * (k + u));
            vv[u] = ld_stream(v + 32 * (k + u));
        }
        XT xx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xx[u] = x(cc[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fma(to_acc<AT>(vv[u]), (AT)xx[u], acc);
    }
    for (; k < w; ++k) {
        int32_t cc = ld_stream(c + 32 * k);
        VT vv = ld_stream(v + 32 * k);
        acc = fma(to_acc<AT>(vv), (AT)x(cc), acc);
    }
    return acc;
}

template <class VT, class XT, class AT, int U = 3, class G>
__device__ __forceinline__ AT slice_spmv_bcrs3(const fe_matrix &A, int64_t s, int lane, const G &x) {
    const int64_t b = A.d_slice_ptr[s];
    const int w = (int)((A.d_slice_ptr[s + 1] - b) >> 5);
    const int32_t *c = A.d_cols + b + lane;
    const VT *v = reinterpret_cast<const VT *>(A.d_vals) + 3 * b + lane;
    AT acc = AT(0);
    int k = 0;
    for (; k + U <= w; k += U) {     // U slots' loads in flight per trip
        int32_t jj[U];
        VT vv[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            jj[u] = ld_stream(c + 32 * (k + u));
#pragma unroll
            for (int t = 0; t < 3; ++t) vv[u][t] = ld_stream(v + 96 * (k + u) + 32 * t);
        }
        XT xx[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int t = 0; t < 3; ++t) xx[u][t] = x((int64_t)jj[u] + t);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int t = 0; t < 3; ++t) acc = fma(to_acc<AT>(vv[u][t]), (AT)xx[u][t], acc);
    }
    for (; k < w; ++k) {
        int32_t j = ld_stream(c + 32 * k);
#pragma unroll
        for (int t = 0; t < 3; ++t)
            acc = fma(to_acc<AT>(ld_stream(v + 96 * k + 32 * t)),
                      (AT)x((int64_t)j + t), acc);
    }
    return acc;
}

// A warp's grid-stride walk over BCRS3 slices s0, s0 + stride, ... in which
// the column indices of the next slice are loaded during the current slice's
// trip.  A slice of nine slots (every 27-point row) then puts its value loads
// and its operand gathers in flight together: one round of memory latency
// per slice, not two (indices, then the gathers that depend on them).  Slices
// of another width take slice_spmv_bcrs3.  The FMA order is
// slice_spmv_bcrs3's, so results are bitwise the same.  out(s, y, x_row)
// receives lane's row sum of slice s and the operand at lane's row.
template <class VT, class XT, class AT, class G, class F>
__device__ __forceinline__ void bcrs3_slices_prefetch(const fe_matrix &A, int64_t s0, int64_t stride,
                                                      int lane, const G &x, F &&out) {
    constexpr int W = 9;
    const int64_t ns = A.n_slices;
    if (s0 >= ns) return;
    const int64_t *sp = A.d_slice_ptr;
    const int32_t *cols = A.d_cols + lane;
    const VT *vals = reinterpret_cast<const VT *>(A.d_vals) + lane;
    int64_t b = sp[s0];
    int w = (int)((sp[s0 + 1] - b) >> 5);
    int32_t jj[W];
#pragma unroll
    for (int u = 0; u < W; ++u) jj[u] = (w == W) ? ld_stream(cols + b + 32 * u) : 0;
    for (int64_t s = s0; s < ns; s += stride) {
        // the next slice's bounds (their latency runs under this trip's loads)
        const int64_t sn = s + stride;
        int64_t bn = 0;
        int wn = 0;
        if (sn < ns) {
            bn = sp[sn];
            wn = (int)((sp[sn + 1] - bn) >> 5);
        }
        const int64_t row = s * kSlice + lane;
        const XT xr = row < A.n_rows ? x(row) : XT(0);   // for out(), loaded with the gathers
        AT acc = AT(0);
        if (w == W) {
            const VT *v = vals + 3 * b;
            VT vv[W][3];
            XT xx[W][3];
#pragma unroll
            for (int u = 0; u < W; ++u)
#pragma unroll
                for (int t = 0; t < 3; ++t) vv[u][t] = ld_stream(v + 96 * u + 32 * t);
#pragma unroll
            for (int u = 0; u < W; ++u)
#pragma unroll
                for (int t = 0; t < 3; ++t) xx[u][t] = x((int64_t)jj[u] + t);
#pragma unroll
            for (int u = 0; u < W; ++u) jj[u] = (wn == W) ? ld_stream(cols + bn + 32 * u) : 0;
#pragma unroll
            for (int u = 0; u < W; ++u)
#pragma unroll
                for (int t = 0; t < 3; ++t) acc = fma(to_acc<AT>(vv[u][t]), (AT)xx[u][t], acc);
        } else {
#pragma unroll
            for (int u = 0; u < W; ++u) jj[u] = (wn == W) ? ld_stream(cols + bn + 32 * u) : 0;
            acc = slice_spmv_bcrs3<VT, XT, AT, W>(A, s, lane, x);
        }
        out(s, acc, xr);
        b = bn;
        w = wn;
    }
}

// CSR: four lanes per row, eight rows per pass, four passes per slice.  Lane
// j of group g runs entries lo + j, lo + j + 4, ... of row 8p + g (one FMA
// per entry slot; the four lanes read 32 contiguous bytes of values per step;
// slots past the row end load nothing and add 0 * 0).
// The four per-pass partials of a lane are then combined across its group by
// a fixed transpose-reduce (xor 1 then xor 2: three adds per lane) and one
// shuffle hands each row's sum to the lane of that row.  The order of every
// addition is fixed, so results are bitwise repeatable.
template <class VT, class XT, class AT, class G>
__device__ __forceinline__ AT slice_spmv_csr(const fe_matrix &A, int64_t s, int lane, const G &x) {
    const int g = lane >> 2, j = lane & 3;
    const int64_t r0 = s * kSlice;
    const int64_t nrows = A.n_rows;
    const VT *vals = reinterpret_cast<const VT *>(A.d_vals);
    AT part[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t row = r0 + 8 * p + g;
        AT acc = AT(0);
        if (row < nrows) {
            const int32_t lo = A.d_row_ptr[row], hi = A.d_row_ptr[row + 1];
            // 28 entries per group per trip (7 per lane, a 27-point row in one
            // trip); every load of the trip is issued before the first FMA
            for (int32_t k = lo + j; k < hi; k += 28) {
                int32_t c[7];
                VT v[7];
#pragma unroll
                for (int u = 0; u < 7; ++u) {
                    const bool ok = k + 4 * u < hi;
                    c[u] = ok ? ld_stream(A.d_cols + k + 4 * u) : 0;
                    v[u] = ok ? ld_stream(vals + k + 4 * u) : VT(0);
                }
                XT xx[7];
#pragma unroll
                for (int u = 0; u < 7; ++u) xx[u] = (k + 4 * u < hi) ? x(c[u]) : XT(0);
#pragma unroll
                for (int u = 0; u < 7; ++u) acc = fma(to_acc<AT>(v[u]), (AT)xx[u], acc);
            }
        }
        part[p] = acc;
    }
    // transpose-reduce over the group: after xor 1 a lane keeps passes
    // {2b, 2b+1} (b = j & 1), after xor 2 pass q = 2b + ((j >> 1) & 1)
    const int b = j & 1, h = (j >> 1) & 1;
    const AT s0 = __shfl_xor_sync(0xffffffffu, b ? part[0] : part[2], 1);
    const AT s1 = __shfl_xor_sync(0xffffffffu, b ? part[1] : part[3], 1);
    const AT k0 = (b ? part[2] : part[0]) + s0;
    const AT k1 = (b ? part[3] : part[1]) + s1;
    const AT t = __shfl_xor_sync(0xffffffffu, h ? k0 : k1, 2);
    const AT row_sum = (h ? k1 : k0) + t;     // sum of row 8 q + g, q = 2b + h
    // lane L takes row L = 8 q + g from lane 4 g + j with q(j) = L / 8
    const int q = lane >> 3;
    const int src = 4 * (lane & 7) + ((q & 1) << 1) + (q >> 1);
    return __shfl_sync(0xffffffffu, row_sum, src);
}

// The paper's BCRS (FE_FMT_VBCRS): the CSR kernel's layout -- four lanes per
// row, eight rows per pass, four passes per 32-row slice -- with a lane
// taking whole segments: lane j of a row's group runs segments lo + j,
// lo + j + 4, lo + j + 8 (a 27-point row has at most nine), reading each
// segment's first column and value offset and its (up to three, then a loop)
// values, which are contiguous in the CSR value array.  Every load of a trip
// is issued before the first FMA; the four lane partials of a row are then
// combined by the same fixed transpose-reduce as the CSR kernel.  S = segments
// per lane per trip: 3 covers a 27-point row (nine segments) in one trip --
// the stand-alone SpMV's choice; the CG kernels, which hold more state, take
// 2 (two trips per row, no spills at their register budgets).
template <class VT, class XT, class AT, int S = 2, class G>
__device__ __forceinline__ AT slice_spmv_vbcrs(const fe_matrix &A, int64_t s, int lane, const G &x) {
    constexpr int L = 3;              // values unrolled per segment
    const int g = lane >> 2, j = lane & 3;
    const int64_t r0 = s * kSlice;
    const int64_t nrows = A.n_rows;
    const VT *vals = reinterpret_cast<const VT *>(A.d_vals);
    const int32_t *seg_ptr = A.d_row_ptr, *jas = A.d_cols, *off = A.d_seg_offsets;
    AT part[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t row = r0 + 8 * p + g;
        AT acc = AT(0);
        if (row < nrows) {
            const int32_t lo = seg_ptr[row], hi = seg_ptr[row + 1];
            for (int32_t q = lo + j; q < hi; q += 4 * S) {
                int32_t c[S], o[S], len[S];
#pragma unroll
                for (int u = 0; u < S; ++u) {
                    const bool ok = q + 4 * u < hi;
                    c[u] = ok ? ld_stream(jas + q + 4 * u) : 0;
                    o[u] = ok ? ld_stream(off + q + 4 * u) : 0;
                    len[u] = ok ? ld_stream(off + q + 4 * u + 1) - o[u] : 0;
                }
                VT v[S][L];
                XT xx[S][L];
#pragma unroll
                for (int u = 0; u < S; ++u)
#pragma unroll
                    for (int t = 0; t < L; ++t) {
                        const bool ok = t < len[u];
                        v[u][t] = ok ? ld_stream(vals + o[u] + t) : VT(0);
                        xx[u][t] = ok ? x((int64_t)c[u] + t) : XT(0);
                    }
#pragma unroll
                for (int u = 0; u < S; ++u) {
#pragma unroll
                    for (int t = 0; t < L; ++t)
                        if (t < len[u]) acc = fma(to_acc<AT>(v[u][t]), (AT)xx[u][t], acc);
                    for (int t = L; t < len[u]; ++t)       // runs longer than three
                        acc = fma(to_acc<AT>(ld_stream(vals + o[u] + t)), (AT)x((int64_t)c[u] + t), acc);
                }
            }
        }
        part[p] = acc;
    }
    const int b = j & 1, h = (j >> 1) & 1;
    const AT s0 = __shfl_xor_sync(0xffffffffu, b ? part[0] : part[2], 1);
    const AT s1 = __shfl_xor_sync(0xffffffffu, b ? part[1] : part[3], 1);
    const AT k0 = (b ? part[2] : part[0]) + s0;
    const AT k1 = (b ? part[3] : part[1]) + s1;
    const AT t = __shfl_xor_sync(0xffffffffu, h ? k0 : k1, 2);
    const AT row_sum = (h ? k1 : k0) + t;
    const int qq = lane >> 3;
    const int src = 4 * (lane & 7) + ((qq & 1) << 1) + (qq >> 1);
    return __shfl_sync(0xffffffffu, row_sum, src);
}

// UN: loads in flight per lane and trip where the format has the choice --
// VBCRS segments (default 2), BCRS3 slots (default 3); 0 takes the default.
template <int FMT, class VT, class XT, class AT, class G, int UN = 0>
__device__ __forceinline__ AT slice_spmv_g(const fe_matrix &A, int64_t s, int lane, const G &x) {
    if constexpr (FMT == FE_FMT_CSR) return slice_spmv_csr<VT, XT, AT>(A, s, lane, x);
    else if constexpr (FMT == FE_FMT_VBCRS) return slice_spmv_vbcrs<VT, XT, AT, UN ? UN : 2>(A, s, lane, x);
    else if constexpr (FMT == FE_FMT_SELL) return slice_spmv_sell<VT, XT, AT>(A, s, lane, x);
    else return slice_spmv_bcrs3<VT, XT, AT, UN ? UN : 3>(A, s, lane, x);
}

template <int FMT, class VT, class XT, class AT, bool kReadOnlyX, int UN = 0>
__device__ __forceinline__ AT slice_spmv(const fe_matrix &A, int64_t s, int lane, const XT *x) {
    return slice_spmv_g<FMT, VT, XT, AT, PtrGather<kReadOnlyX, XT>, UN>(A, s, lane, PtrGather<kReadOnlyX, XT>{x});
}

}  // namespace fe
