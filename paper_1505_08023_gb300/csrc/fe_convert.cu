// fe_convert.cu -- conversion of the assembled CSR matrix into the sliced
// formats used by the solver (paper Sec. 3.1: keep CRS for generation and
// assembly, convert at the start of CG).
//
//   SELL  : 32-row slices, column-major inside a slice, each slice padded to
//           its longest row (padding: value 0, column = the row's last column).
//   BCRS3 : the paper's 1 x n segments (runs of adjacent columns, Sec. 3.1)
//           with every segment stored as a fixed 1 x 3 block: one column
//           index per three values, no offsets array, no length switch
//           (Fig 3.3 unrolls lengths 1..4; a fixed length needs no branch).
//           Segments are greedy: a segment starts at the first column of the
//           row not yet covered and takes that column and the next two.
#include "fe_common.cuh"

namespace fe {

// Number of 1x3 segments the greedy rule makes for a sorted column list.
__device__ __forceinline__ int bcrs3_segments(const int32_t *cols, int32_t lo, int32_t hi) {
    int n = 0;
    int32_t j = lo;
    while (j < hi) {
        const int32_t c = cols[j];
        ++n;
        while (j < hi && cols[j] <= c + 2) ++j;
    }
    return n;
}

// Slot count (32 x widest row) of every slice, written to slice_ptr[s + 1].
template <int FMT>
__global__ void k_slice_widths(int64_t n_rows, int64_t n_slices, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ cols, int64_t *__restrict__ slice_ptr) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < n_slices;
         s += warps) {
        const int64_t row = s * kSlice + lane;
        int w = 0;
        if (row < n_rows) {
            const int32_t lo = row_ptr[row], hi = row_ptr[row + 1];
            w = (FMT == FE_FMT_SELL) ? (hi - lo) : bcrs3_segments(cols, lo, hi);
        }
        w = warp_max(w);
        if (lane == 0) slice_ptr[s + 1] = (int64_t)w * kSlice;
    }
}

// In-place inclusive scan of a[1..n] with a[0] = 0, one block of 1024
// threads (each thread scans a contiguous chunk; chunk totals are scanned in
// shared memory).  n is at most a few million slices.
__global__ void __launch_bounds__(1024) k_scan_slices(int64_t n, int64_t *__restrict__ a) {
    __shared__ int64_t tot[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t lo = 1 + t * chunk;
    const int64_t hi = (lo + chunk - 1 < n) ? lo + chunk : n + 1;
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a[i];
    tot[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v = (t >= o) ? tot[t - o] : 0;
        __syncthreads();
        tot[t] += v;
        __syncthreads();
    }
    int64_t run = (t == 0) ? 0 : tot[t - 1];
    for (int64_t i = lo; i < hi; ++i) {
        run += a[i];
        a[i] = run;
    }
    if (t == 0) a[0] = 0;
}

template <class VT> __device__ __forceinline__ VT round_to(double v);
template <> __device__ __forceinline__ double round_to<double>(double v) { return v; }
template <> __device__ __forceinline__ float round_to<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 round_to<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);  // round to nearest even
}

template <class VT>
__global__ void k_fill_sell(int64_t n_rows, int64_t n_slices, const int32_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ cols, const double *__restrict__ vals,
                            const int64_t *__restrict__ slice_ptr, int32_t *__restrict__ out_cols,
                            VT *__restrict__ out_vals) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < n_slices;
         s += warps) {
        const int64_t row = s * kSlice + lane;
        const int64_t base = slice_ptr[s];
        const int w = (int)((slice_ptr[s + 1] - base) >> 5);
        int32_t lo = 0, hi = 0, pad_col = 0;
        if (row < n_rows) {
            lo = row_ptr[row];
            hi = row_ptr[row + 1];
            pad_col = (hi > lo) ? cols[hi - 1] : (int32_t)row;
        }
        for (int k = 0; k < w; ++k) {
            const int64_t slot = base + (int64_t)k * kSlice + lane;
            if (lo + k < hi) {
                out_cols[slot] = cols[lo + k];
                out_vals[slot] = round_to<VT>(vals[lo + k]);
            } else {
                out_cols[slot] = pad_col;
                out_vals[slot] = round_to<VT>(0.0);
            }
        }
    }
}

// One warp per slice.  The slice's CSR entries are contiguous; when they fit
// (kFillCap: 32 rows of 27) the warp first copies them to shared memory with
// coalesced loads, so that each lane's walk along its own row (a 27-entry
// stride between lanes) reads shared memory instead of scattered global
// sectors; longer slices read global memory directly.
constexpr int kFillWarps = 4;
constexpr int kFillCap = 32 * 27;

template <class VT>
__global__ void __launch_bounds__(32 * kFillWarps)
k_fill_bcrs3(int64_t n_rows, int64_t n_cols, int64_t n_slices,
             const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ cols,
             const double *__restrict__ vals, const int64_t *__restrict__ slice_ptr,
             int32_t *__restrict__ out_cols, VT *__restrict__ out_vals) {
    __shared__ int32_t s_cols[kFillWarps][kFillCap];
    __shared__ double s_vals[kFillWarps][kFillCap];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * kFillWarps;
    const int32_t cmax = (int32_t)(n_cols - 3);  // last legal segment start
    for (int64_t s = blockIdx.x * (int64_t)kFillWarps + wib; s < n_slices; s += warps) {
        const int64_t row = s * kSlice + lane;
        const int64_t base = slice_ptr[s];
        const int w = (int)((slice_ptr[s + 1] - base) >> 5);
        const int64_t last = (s * kSlice + kSlice < n_rows) ? s * kSlice + kSlice : n_rows;
        const int32_t lo0 = row_ptr[s * kSlice], hi0 = row_ptr[last];
        const bool staged = hi0 - lo0 <= kFillCap;
        if (staged) {
            for (int32_t t = lane; t < hi0 - lo0; t += 32) {
                s_cols[wib][t] = cols[lo0 + t];
                s_vals[wib][t] = vals[lo0 + t];
            }
        }
        __syncwarp();
        int32_t j = 0, hi = 0, last_start = 0;
        if (row < n_rows) {
            j = row_ptr[row];
            hi = row_ptr[row + 1];
        }
        auto col_at = [&](int32_t jj) { return staged ? s_cols[wib][jj - lo0] : cols[jj]; };
        auto val_at = [&](int32_t jj) { return staged ? s_vals[wib][jj - lo0] : vals[jj]; };
        for (int k = 0; k < w; ++k) {
            const int64_t slot = base + (int64_t)k * kSlice + lane;
            VT *v = out_vals + 3 * base + (int64_t)k * 96 + lane;
            double seg[3] = {0.0, 0.0, 0.0};
            int32_t start = last_start;
            if (j < hi) {
                const int32_t c = col_at(j);
                // shift the block left when it would run past the last column
                start = c < cmax ? c : cmax;
                while (j < hi && col_at(j) <= c + 2) {
                    seg[col_at(j) - start] = val_at(j);
                    ++j;
                }
                last_start = start;
            }
            out_cols[slot] = start;
#pragma unroll
            for (int t = 0; t < 3; ++t) v[32 * t] = round_to<VT>(seg[t]);
        }
        __syncwarp();   // the slice buffer is reused by the warp's next slice
    }
}

template <class VT>
__global__ void k_round(int64_t n, const double *__restrict__ src, VT *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = round_to<VT>(src[i]);
}

static int warp_grid(int64_t n_slices, int warps_per_block = 8) {
    int64_t blocks = (n_slices + warps_per_block - 1) / warps_per_block;
    int64_t cap = (int64_t)sm_count() * 16;
    if (cap < 1) cap = 1024;
    return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

template <class VT>
static fe_status launch_fill(const fe_matrix *src, const fe_matrix *dst, cudaStream_t s) {
    if (dst->format == FE_FMT_SELL)
        k_fill_sell<VT><<<warp_grid(dst->n_slices), 256, 0, s>>>(
            src->n_rows, dst->n_slices, src->d_row_ptr, src->d_cols, (const double *)src->d_vals,
            dst->d_slice_ptr, const_cast<int32_t *>(dst->d_cols), (VT *)const_cast<void *>(dst->d_vals));
    else
        k_fill_bcrs3<VT><<<warp_grid(dst->n_slices, kFillWarps), 32 * kFillWarps, 0, s>>>(
            src->n_rows, src->n_cols, dst->n_slices, src->d_row_ptr, src->d_cols,
            (const double *)src->d_vals, dst->d_slice_ptr, const_cast<int32_t *>(dst->d_cols),
            (VT *)const_cast<void *>(dst->d_vals));
    FE_TRY_LAUNCH();
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_sliced_plan(int32_t format, int64_t n_rows, int64_t n_cols, const int32_t *d_row_ptr,
                         const int32_t *d_cols, int64_t *d_slice_ptr, int64_t *h_n_stored,
                         fe_stream_t stream) {
    if ((format != FE_FMT_SELL && format != FE_FMT_BCRS3) || n_rows < 1 || n_cols < 1 ||
        !d_row_ptr || !d_cols || !d_slice_ptr || !h_n_stored || !aligned(d_slice_ptr, 8))
        return FE_ERR_ARG;
    if (format == FE_FMT_BCRS3 && n_cols < 3) return FE_ERR_ARG;
    if (n_rows > INT32_MAX || n_cols > INT32_MAX) return FE_ERR_OVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ns = (n_rows + kSlice - 1) / kSlice;
    if (format == FE_FMT_SELL)
        k_slice_widths<FE_FMT_SELL><<<warp_grid(ns), 256, 0, s>>>(n_rows, ns, d_row_ptr, d_cols, d_slice_ptr);
    else
        k_slice_widths<FE_FMT_BCRS3><<<warp_grid(ns), 256, 0, s>>>(n_rows, ns, d_row_ptr, d_cols, d_slice_ptr);
    FE_TRY_LAUNCH();
    k_scan_slices<<<1, 1024, 0, s>>>(ns, d_slice_ptr);
    FE_TRY_LAUNCH();
    int64_t total = 0;
    FE_TRY_CUDA(cudaMemcpyAsync(&total, d_slice_ptr + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    *h_n_stored = total;
    return FE_OK;
}

fe_status fe_convert(const fe_matrix *src, const fe_matrix *dst, fe_stream_t stream) {
    fe_status st = check_matrix(src);
    if (st != FE_OK) return st;
    st = check_matrix(dst);
    if (st != FE_OK) return st;
    if (src->format != FE_FMT_CSR || src->value_type != FE_VAL_F64) return FE_ERR_ARG;
    if (dst->format == FE_FMT_CSR) return FE_ERR_ARG;
    if (dst->n_rows != src->n_rows || dst->n_cols != src->n_cols) return FE_ERR_ARG;
    if (!aligned(dst->d_vals, 8) || !aligned(dst->d_cols, 4)) return FE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (dst->value_type) {
        case FE_VAL_F64: return launch_fill<double>(src, dst, s);
        case FE_VAL_F32: return launch_fill<float>(src, dst, s);
        default: return launch_fill<__nv_bfloat16>(src, dst, s);
    }
}

fe_status fe_round_values(int64_t n, const double *d_src, int32_t value_type, void *d_dst,
                          fe_stream_t stream) {
    if (n < 0 || !d_src || !d_dst || (value_type != FE_VAL_F32 && value_type != FE_VAL_BF16))
        return FE_ERR_ARG;
    if (n == 0) return FE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t blocks = (n + 255) / 256, cap = (int64_t)sm_count() * 16;
    if (cap < 1) cap = 1024;
    int grid = (int)(blocks > cap ? cap : blocks);
    if (value_type == FE_VAL_F32) k_round<float><<<grid, 256, 0, s>>>(n, d_src, (float *)d_dst);
    else k_round<__nv_bfloat16><<<grid, 256, 0, s>>>(n, d_src, (__nv_bfloat16 *)d_dst);
    FE_TRY_LAUNCH();
    return FE_OK;
}

}  // extern "C"
