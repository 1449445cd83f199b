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

// Shared-memory staging for the CSR slice kernel: values and gathered vector
// entries of one warp's 32 rows, in chunks of kCsrStage entries.
constexpr int kCsrStage = 32 * 27;

// One warp computes the 32 rows of slice s; returns lane's row sum (0 for
// rows past the end).  XT: vector type, AT: accumulation type.
template <class VT, class XT, class AT, bool kReadOnlyX>
__device__ __forceinline__ AT slice_spmv_sell(const fe_matrix &A, int64_t s, int lane,
                                              const XT *x) {
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
        for (int u = 0; u < U; ++u) xx[u] = ld_vec<kReadOnlyX>(x + cc[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc = fma(to_acc<AT>(vv[u]), (AT)xx[u], acc);
    }
    for (; k < w; ++k) {
        int32_t cc = ld_stream(c + 32 * k);
        VT vv = ld_stream(v + 32 * k);
        acc = fma(to_acc<AT>(vv), (AT)ld_vec<kReadOnlyX>(x + cc), acc);
    }
    return acc;
}

template <class VT, class XT, class AT, bool kReadOnlyX>
__device__ __forceinline__ AT slice_spmv_bcrs3(const fe_matrix &A, int64_t s, int lane,
                                               const XT *x) {
    const int64_t b = A.d_slice_ptr[s];
    const int w = (int)((A.d_slice_ptr[s + 1] - b) >> 5);
    const int32_t *c = A.d_cols + b + lane;
    const VT *v = reinterpret_cast<const VT *>(A.d_vals) + 3 * b + lane;
    AT acc = AT(0);
    int k = 0;
    constexpr int U = 3;
    for (; k + U <= w; k += U) {
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
            for (int t = 0; t < 3; ++t) xx[u][t] = ld_vec<kReadOnlyX>(x + jj[u] + t);
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
                      (AT)ld_vec<kReadOnlyX>(x + j + t), acc);
    }
    return acc;
}

// CSR: the warp stages its rows' values and gathered x entries in shared
// memory with coalesced loads, then each lane runs its own row sequentially
// (one FMA per entry, all lanes busy).  sv/sx: kCsrStage entries per warp.
template <class VT, class XT, class AT, bool kReadOnlyX>
__device__ __forceinline__ AT slice_spmv_csr(const fe_matrix &A, int64_t s, int lane,
                                             const XT *x, AT *sv, AT *sx) {
    const int64_t r0 = s * kSlice;
    const int64_t nrows = A.n_rows;
    const int64_t row = r0 + lane;
    const int64_t last = (r0 + kSlice < nrows) ? r0 + kSlice : nrows;
    const int32_t base = A.d_row_ptr[r0];
    const int32_t end = A.d_row_ptr[last];
    int32_t my_lo = 0, my_hi = 0;
    if (row < nrows) {
        my_lo = A.d_row_ptr[row];
        my_hi = A.d_row_ptr[row + 1];
    }
    const VT *vals = reinterpret_cast<const VT *>(A.d_vals);
    AT acc = AT(0);
    for (int32_t c0 = base; c0 < end; c0 += kCsrStage) {
        const int32_t cn = (end - c0 < kCsrStage) ? end - c0 : kCsrStage;
        for (int32_t t = lane; t < cn; t += 32) {
            const int32_t col = ld_stream(A.d_cols + c0 + t);
            sv[t] = to_acc<AT>(ld_stream(vals + c0 + t));
            sx[t] = (AT)ld_vec<kReadOnlyX>(x + col);
        }
        __syncwarp();
        const int32_t lo = (my_lo > c0) ? my_lo : c0;
        const int32_t hi = (my_hi < c0 + cn) ? my_hi : c0 + cn;
        for (int32_t k = lo; k < hi; ++k) acc = fma(sv[k - c0], sx[k - c0], acc);
        __syncwarp();
    }
    return acc;
}

template <int FMT, class VT, class XT, class AT, bool kReadOnlyX>
__device__ __forceinline__ AT slice_spmv(const fe_matrix &A, int64_t s, int lane,
                                         const XT *x, AT *sv, AT *sx) {
    if constexpr (FMT == FE_FMT_CSR) return slice_spmv_csr<VT, XT, AT, kReadOnlyX>(A, s, lane, x, sv, sx);
    else if constexpr (FMT == FE_FMT_SELL) return slice_spmv_sell<VT, XT, AT, kReadOnlyX>(A, s, lane, x);
    else return slice_spmv_bcrs3<VT, XT, AT, kReadOnlyX>(A, s, lane, x);
}

// Dynamic shared memory a block of `warps` warps needs for format FMT.
template <int FMT, class AT> constexpr size_t spmv_smem_bytes(int warps) {
    return FMT == FE_FMT_CSR ? (size_t)warps * 2 * kCsrStage * sizeof(AT) : 0;
}

}  // namespace fe
