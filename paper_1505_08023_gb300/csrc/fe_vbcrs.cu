// fe_vbcrs.cu -- the paper's BCRS (Sec. 3.1, Fig 3.2/3.3) on the GPU: the
// CSR matrix's entries grouped into maximal runs of adjacent columns
// ("segments"), described by a row pointer over segments (ptr), each
// segment's first column (jas) and first value (offsets); the values stay the
// CSR array.  This file builds those arrays from a CSR matrix; the SpMV is
// slice_spmv_vbcrs in fe_common.cuh.
//
// A segment starts at the first entry of a row and wherever a column is not
// the previous column + 1 (columns are sorted).  Counting, scanning and
// filling are one thread per row; the scan is two-level (per-block sums,
// one block over the block sums, then the per-block scan with its offset).
#include "fe_common.cuh"

namespace fe {

constexpr int kVbThreads = 1024;

__device__ __forceinline__ int32_t row_segments(const int32_t *row_ptr, const int32_t *cols, int64_t row) {
    const int32_t lo = row_ptr[row], hi = row_ptr[row + 1];
    int32_t n = hi > lo ? 1 : 0;
    for (int32_t k = lo + 1; k < hi; ++k) n += cols[k] != cols[k - 1] + 1;
    return n;
}

// inclusive scan of one value per thread over the block (warp shuffles, then
// the warp totals through shared memory); returns the thread's inclusive sum
__device__ __forceinline__ int64_t block_inclusive_scan(int64_t v, int64_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int64_t r = v + (warp > 0 ? s_warp[warp - 1] : 0);
    __syncthreads();                     // s_warp is reused by the caller's next scan
    return r;
}

// 1: segments of the block's rows, summed per block
__global__ void __launch_bounds__(kVbThreads) k_vb_block_sums(int64_t m, const int32_t *__restrict__ row_ptr,
                                                              const int32_t *__restrict__ cols,
                                                              int64_t *__restrict__ block_sum) {
    __shared__ int64_t s_warp[32];
    const int64_t row = (int64_t)blockIdx.x * kVbThreads + threadIdx.x;
    const int64_t n = row < m ? row_segments(row_ptr, cols, row) : 0;
    const int64_t incl = block_inclusive_scan(n, s_warp);
    if (threadIdx.x == kVbThreads - 1) block_sum[blockIdx.x] = incl;
}

// 2: exclusive scan of the block sums (one block, chunks of kVbThreads)
__global__ void __launch_bounds__(kVbThreads) k_vb_scan_blocks(int64_t nb, int64_t *__restrict__ block_sum,
                                                               int64_t *__restrict__ total) {
    __shared__ int64_t s_warp[32];
    int64_t base = 0;
    for (int64_t c = 0; c < nb; c += kVbThreads) {
        const int64_t i = c + threadIdx.x;
        const int64_t v = i < nb ? block_sum[i] : 0;
        const int64_t incl = block_inclusive_scan(v, s_warp);
        if (i < nb) block_sum[i] = base + incl - v;
        __shared__ int64_t s_last;
        if (threadIdx.x == kVbThreads - 1) s_last = incl;
        __syncthreads();
        base += s_last;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = base;
}

// 3: segment row pointer = block offset + exclusive scan inside the block
__global__ void __launch_bounds__(kVbThreads) k_vb_seg_ptr(int64_t m, const int32_t *__restrict__ row_ptr,
                                                           const int32_t *__restrict__ cols,
                                                           const int64_t *__restrict__ block_off,
                                                           const int64_t *__restrict__ total,
                                                           int32_t *__restrict__ seg_ptr) {
    __shared__ int64_t s_warp[32];
    const int64_t row = (int64_t)blockIdx.x * kVbThreads + threadIdx.x;
    const int64_t n = row < m ? row_segments(row_ptr, cols, row) : 0;
    const int64_t incl = block_inclusive_scan(n, s_warp);
    if (row < m) seg_ptr[row] = (int32_t)(block_off[blockIdx.x] + incl - n);
    if (row == 0) seg_ptr[m] = (int32_t)*total;
}

// jas and offsets, one thread per row
__global__ void k_vb_fill(int64_t m, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ cols,
                          const int32_t *__restrict__ seg_ptr, int32_t *__restrict__ jas,
                          int32_t *__restrict__ offsets) {
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < m;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lo = row_ptr[row], hi = row_ptr[row + 1];
        int32_t s = seg_ptr[row];
        for (int32_t k = lo; k < hi; ++k) {
            if (k == lo || cols[k] != cols[k - 1] + 1) {
                jas[s] = cols[k];
                offsets[s] = k;
                ++s;
            }
        }
        if (row == m - 1) offsets[s] = hi;   // offsets[nns] = nnz
    }
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_vbcrs_workspace(int64_t n_rows, size_t *h_bytes) {
    if (n_rows < 1 || !h_bytes) return FE_ERR_ARG;
    const int64_t nb = (n_rows + kVbThreads - 1) / kVbThreads;
    *h_bytes = (size_t)(nb + 1) * sizeof(int64_t);
    return FE_OK;
}

fe_status fe_vbcrs_plan(const fe_matrix *csr, int32_t *d_seg_ptr, void *d_work, size_t work_bytes,
                        int64_t *h_nns, fe_stream_t stream) {
    fe_status st = check_matrix(csr);
    if (st != FE_OK) return st;
    if (csr->format != FE_FMT_CSR || !d_seg_ptr || !d_work || !h_nns || !aligned(d_seg_ptr, 4) ||
        !aligned(d_work, 8))
        return FE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = csr->n_rows;
    const int64_t nb = (m + kVbThreads - 1) / kVbThreads;
    if (work_bytes < (size_t)(nb + 1) * sizeof(int64_t)) return FE_ERR_WORKSPACE;
    int64_t *tmp = (int64_t *)d_work;             // nb block sums, then the total
    k_vb_block_sums<<<(unsigned)nb, kVbThreads, 0, s>>>(m, csr->d_row_ptr, csr->d_cols, tmp);
    FE_TRY_LAUNCH();
    k_vb_scan_blocks<<<1, kVbThreads, 0, s>>>(nb, tmp, tmp + nb);
    FE_TRY_LAUNCH();
    k_vb_seg_ptr<<<(unsigned)nb, kVbThreads, 0, s>>>(m, csr->d_row_ptr, csr->d_cols, tmp, tmp + nb, d_seg_ptr);
    FE_TRY_LAUNCH();
    int64_t total = 0;
    FE_TRY_CUDA(cudaMemcpyAsync(&total, tmp + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    if (total > INT32_MAX) return FE_ERR_OVERFLOW;
    *h_nns = total;
    return FE_OK;
}

fe_status fe_vbcrs_fill(const fe_matrix *csr, const int32_t *d_seg_ptr, int32_t *d_jas,
                        int32_t *d_seg_offsets, fe_stream_t stream) {
    fe_status st = check_matrix(csr);
    if (st != FE_OK) return st;
    if (csr->format != FE_FMT_CSR || !d_seg_ptr || !d_jas || !d_seg_offsets) return FE_ERR_ARG;
    if (!aligned(d_seg_ptr, 4) || !aligned(d_jas, 4) || !aligned(d_seg_offsets, 4)) return FE_ERR_ARG;
    const int64_t m = csr->n_rows;
    int64_t blocks = (m + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    k_vb_fill<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, (cudaStream_t)stream>>>(
        m, csr->d_row_ptr, csr->d_cols, d_seg_ptr, d_jas, d_seg_offsets);
    FE_TRY_LAUNCH();
    return FE_OK;
}

}  // extern "C"
