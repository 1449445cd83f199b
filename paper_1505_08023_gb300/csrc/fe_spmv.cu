// fe_spmv.cu -- stand-alone SpMV y = A x (paper Fig 3.1 CRS, Fig 3.2/3.3 BCRS)
// in every storage format and value type.  One warp per 32-row slice,
// grid-stride over slices so that the blocks in flight cover a narrow band of
// rows and the gathered x entries (three planes of the mesh) stay in L2.
#include "fe_common.cuh"

namespace fe {

constexpr int kSpmvWarps = 8;

template <int FMT, class VT, class XT, class AT>
__global__ void __launch_bounds__(kSpmvWarps * 32)
k_spmv(const fe_matrix A, const XT *__restrict__ x, XT *__restrict__ y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tw = (int64_t)gridDim.x * kSpmvWarps;
    for (int64_t s = (int64_t)blockIdx.x * kSpmvWarps + warp; s < A.n_slices; s += tw) {
        // VBCRS: three segments per lane and trip (one trip per 27-point row)
        const AT v = slice_spmv<FMT, VT, XT, AT, true, FMT == FE_FMT_VBCRS ? 3 : 0>(A, s, lane, x);
        const int64_t row = s * kSlice + lane;
        if (row < A.n_rows) y[row] = (XT)v;
    }
}

template <int FMT, class VT, class XT, class AT>
static fe_status launch(const fe_matrix &A, const XT *x, XT *y, cudaStream_t s) {
    auto kern = k_spmv<FMT, VT, XT, AT>;
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSpmvWarps * 32, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (A.n_slices + kSpmvWarps - 1) / kSpmvWarps;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (cap > 0 && blocks > cap) blocks = cap;
    kern<<<(int)blocks, kSpmvWarps * 32, 0, s>>>(A, x, y);
    FE_TRY_LAUNCH();
    return FE_OK;
}

template <class XT, class AT>
static fe_status dispatch(const fe_matrix *A, const XT *x, XT *y, fe_stream_t stream) {
    fe_status st = check_matrix(A);
    if (st != FE_OK) return st;
    if (x == nullptr || y == nullptr || !aligned(x, sizeof(XT)) || !aligned(y, sizeof(XT))) return FE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    switch (A->format * 3 + A->value_type) {
        case FE_FMT_CSR * 3 + FE_VAL_F64: return launch<FE_FMT_CSR, double, XT, AT>(*A, x, y, s);
        case FE_FMT_CSR * 3 + FE_VAL_F32: return launch<FE_FMT_CSR, float, XT, AT>(*A, x, y, s);
        case FE_FMT_CSR * 3 + FE_VAL_BF16: return launch<FE_FMT_CSR, __nv_bfloat16, XT, AT>(*A, x, y, s);
        case FE_FMT_SELL * 3 + FE_VAL_F64: return launch<FE_FMT_SELL, double, XT, AT>(*A, x, y, s);
        case FE_FMT_SELL * 3 + FE_VAL_F32: return launch<FE_FMT_SELL, float, XT, AT>(*A, x, y, s);
        case FE_FMT_SELL * 3 + FE_VAL_BF16: return launch<FE_FMT_SELL, __nv_bfloat16, XT, AT>(*A, x, y, s);
        case FE_FMT_BCRS3 * 3 + FE_VAL_F64: return launch<FE_FMT_BCRS3, double, XT, AT>(*A, x, y, s);
        case FE_FMT_BCRS3 * 3 + FE_VAL_F32: return launch<FE_FMT_BCRS3, float, XT, AT>(*A, x, y, s);
        case FE_FMT_BCRS3 * 3 + FE_VAL_BF16: return launch<FE_FMT_BCRS3, __nv_bfloat16, XT, AT>(*A, x, y, s);
        case FE_FMT_VBCRS * 3 + FE_VAL_F64: return launch<FE_FMT_VBCRS, double, XT, AT>(*A, x, y, s);
        case FE_FMT_VBCRS * 3 + FE_VAL_F32: return launch<FE_FMT_VBCRS, float, XT, AT>(*A, x, y, s);
        case FE_FMT_VBCRS * 3 + FE_VAL_BF16: return launch<FE_FMT_VBCRS, __nv_bfloat16, XT, AT>(*A, x, y, s);
        default: return FE_ERR_ARG;
    }
}

}  // namespace fe

extern "C" {

fe_status fe_spmv(const fe_matrix *A, const double *d_x, double *d_y, fe_stream_t stream) {
    return fe::dispatch<double, double>(A, d_x, d_y, stream);
}

fe_status fe_spmv_f32(const fe_matrix *A, const float *d_x, float *d_y, fe_stream_t stream) {
    return fe::dispatch<float, float>(A, d_x, d_y, stream);
}

}  // extern "C"
