// fe_mesh.cu -- library status plumbing, problem sizes and the mesh kernel
// (paper Sec. 1: problem domain and mesh processing module).
#include <cstdio>
#include <mutex>

#include "fe_common.cuh"

namespace fe {

static thread_local int g_last_cuda_error = 0;

void set_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

int sm_count() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cached[dev] = n;
    }
    return cached[dev];
}

fe_status check_matrix(const fe_matrix *A) {
    if (A == nullptr || A->n_rows < 1 || A->n_cols < 1 || A->d_cols == nullptr ||
        A->d_vals == nullptr)
        return FE_ERR_ARG;
    if (A->value_type < FE_VAL_F64 || A->value_type > FE_VAL_BF16) return FE_ERR_ARG;
    if (A->n_slices != (A->n_rows + kSlice - 1) / kSlice) return FE_ERR_ARG;
    if (A->n_cols > INT32_MAX - 64 || A->n_rows > INT32_MAX - 64) return FE_ERR_OVERFLOW;
    switch (A->format) {
        case FE_FMT_CSR:
            if (A->d_row_ptr == nullptr || A->n_stored > INT32_MAX) return FE_ERR_ARG;
            break;
        case FE_FMT_SELL:
            if (A->d_slice_ptr == nullptr) return FE_ERR_ARG;
            break;
        case FE_FMT_BCRS3:
            if (A->d_slice_ptr == nullptr || A->n_cols < 3) return FE_ERR_ARG;
            break;
        case FE_FMT_VBCRS:
            if (A->d_row_ptr == nullptr || A->d_seg_offsets == nullptr || A->n_stored > INT32_MAX)
                return FE_ERR_ARG;
            break;
        default:
            return FE_ERR_ARG;
    }
    return FE_OK;
}

// Coordinates (ix/nx, iy/ny, iz/nz), boundary flag and prescribed value of
// every node; one thread per node.
__global__ void k_mesh_nodes(int nx, int ny, int nz, const double *__restrict__ face,
                             double *__restrict__ coords, uint8_t *__restrict__ flag,
                             double *__restrict__ gval) {
    const int64_t nxn = nx + 1, nyn = ny + 1;
    const int64_t m = nxn * nyn * (nz + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nxn);
        const int64_t q = i / nxn;
        const int iy = (int)(q % nyn);
        const int iz = (int)(q / nyn);
        if (coords != nullptr) {
            coords[3 * i + 0] = (double)ix / (double)nx;
            coords[3 * i + 1] = (double)iy / (double)ny;
            coords[3 * i + 2] = (double)iz / (double)nz;
        }
        const bool bnd = ix == 0 || ix == nx || iy == 0 || iy == ny || iz == 0 || iz == nz;
        flag[i] = bnd ? 1 : 0;
        double g = 0.0;
        if (face == nullptr) {
            g = (ix == nx) ? 1.0 : 0.0;
        } else if (bnd) {
            const int64_t fx = nyn * (nz + 1), fy = nxn * (nz + 1);
            const int64_t o_x1 = fx, o_y0 = 2 * fx, o_y1 = 2 * fx + fy, o_z0 = 2 * fx + 2 * fy;
            const int64_t o_z1 = o_z0 + nxn * nyn;
            // faces in order x0, x1, y0, y1, z0, z1: the last one that holds the node wins
            if (iz == nz) g = face[o_z1 + ix + nxn * iy];
            else if (iz == 0) g = face[o_z0 + ix + nxn * iy];
            else if (iy == ny) g = face[o_y1 + ix + nxn * iz];
            else if (iy == 0) g = face[o_y0 + ix + nxn * iz];
            else if (ix == nx) g = face[o_x1 + iy + nyn * iz];
            else g = face[iy + nyn * iz];
        }
        gval[i] = g;
    }
}

// Element connectivity in the local hex8 order; one thread per element.
__global__ void k_mesh_conn(int nx, int ny, int nz, int32_t *__restrict__ conn) {
    const int64_t ne = (int64_t)nx * ny * nz;
    const int64_t nxn = nx + 1, plane = nxn * (ny + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ex = (int)(e % nx);
        const int64_t q = e / nx;
        const int ey = (int)(q % ny);
        const int ez = (int)(q / ny);
        const int64_t n0 = ex + nxn * (ey + (int64_t)(ny + 1) * ez);
        int4 lo = make_int4((int)n0, (int)(n0 + 1), (int)(n0 + 1 + nxn), (int)(n0 + nxn));
        int4 hi = make_int4((int)(n0 + plane), (int)(n0 + plane + 1), (int)(n0 + plane + 1 + nxn),
                            (int)(n0 + plane + nxn));
        reinterpret_cast<int4 *>(conn)[2 * e] = lo;
        reinterpret_cast<int4 *>(conn)[2 * e + 1] = hi;
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t blocks = (n + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * 16;
    if (cap < 1) cap = 1024;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace fe

using namespace fe;

extern "C" {

int fe_last_cuda_error(void) { return fe::g_last_cuda_error; }

const char *fe_version(void) { return "libfe 0.1 (sm_103a)"; }

fe_status fe_problem_sizes(int nx, int ny, int nz, fe_sizes *out) {
    if (out == nullptr || nx < 1 || ny < 1 || nz < 1) return FE_ERR_ARG;
    const int64_t m = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    const int64_t nnz = (int64_t)(3 * (int64_t)nx + 1) * (3 * (int64_t)ny + 1) * (3 * (int64_t)nz + 1);
    out->n_rows = m;
    out->n_elems = (int64_t)nx * ny * nz;
    out->nnz = nnz;
    out->n_faces = 2 * ((int64_t)(ny + 1) * (nz + 1) + (int64_t)(nx + 1) * (nz + 1) +
                        (int64_t)(nx + 1) * (ny + 1));
    out->n_slices = (m + kSlice - 1) / kSlice;
    if (nnz > INT32_MAX || m > INT32_MAX) return FE_ERR_OVERFLOW;
    return FE_OK;
}

fe_status fe_generate_mesh(int nx, int ny, int nz, const double *d_face_vals, double *d_coords,
                           uint8_t *d_bc_flag, double *d_bc_val, int32_t *d_conn,
                           fe_stream_t stream) {
    fe_sizes sz;
    fe_status st = fe_problem_sizes(nx, ny, nz, &sz);
    // the CSR form's nnz limit does not bind the mesh; int32 node ids do
    if (st == FE_ERR_OVERFLOW && (d_conn == nullptr || sz.n_rows <= INT32_MAX)) st = FE_OK;
    if (st != FE_OK) return st;
    if (d_bc_flag == nullptr || d_bc_val == nullptr) return FE_ERR_ARG;
    if ((d_coords && !aligned(d_coords, 8)) || !aligned(d_bc_val, 8) || (d_face_vals && !aligned(d_face_vals, 8)))
        return FE_ERR_ARG;
    if (d_conn != nullptr && !aligned(d_conn, 16)) return FE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_mesh_nodes<<<grid_for(sz.n_rows, 256), 256, 0, s>>>(nx, ny, nz, d_face_vals, d_coords,
                                                          d_bc_flag, d_bc_val);
    FE_TRY_LAUNCH();
    if (d_conn != nullptr) {
        k_mesh_conn<<<grid_for(sz.n_elems, 256), 256, 0, s>>>(nx, ny, nz, d_conn);
        FE_TRY_LAUNCH();
    }
    return FE_OK;
}

}  // extern "C"
