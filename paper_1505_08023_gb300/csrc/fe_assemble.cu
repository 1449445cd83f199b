// fe_assemble.cu -- matrix generation (paper Fig 3.6), element operator and
// FE assembly (paper Sec. 1, Fig 3.7) with the Dirichlet rows, on the GPU.
//
// Design (GB300): the paper's assembly loops over elements and scatters into
// the CRS arrays inside an OpenMP critical section.  Here
//   1. k_element_matrices: one thread per element computes its 8x8 matrix by
//      2x2x2 Gauss quadrature from the node coordinates and stores the 36
//      entries of the upper triangle (SoA, coalesced) in the workspace; a
//      parallelepiped (constant Jacobian) takes the same quadrature with the
//      sum over the points done ahead of time (216 FMAs instead of ~2,000);
//   2. k_assemble_rows: one thread per node gathers the rows of its (up to 8)
//      incident elements in element-id order, so each entry is summed in a
//      fixed order with no atomics, applies the Dirichlet elimination, and
//      writes its CSR row.  The row pointer is the closed-form prefix sum of
//      the per-axis neighbour counts (2 at an end of an axis, 3 inside).
#include "fe_common.cuh"

namespace fe {

// Local hex8 corner order (0,0,0),(1,0,0),(1,1,0),(0,1,0),(0,0,1),(1,0,1),(1,1,1),(0,1,1).
__host__ __device__ constexpr int corner_x(int a) { return (a & 3) == 1 || (a & 3) == 2; }
__host__ __device__ constexpr int corner_y(int a) { return (a & 3) >= 2; }
__host__ __device__ constexpr int corner_z(int a) { return a >= 4; }
__host__ __device__ constexpr int corner_of(int ox, int oy, int oz) {
    return 4 * oz + (oy ? (ox ? 2 : 3) : (ox ? 1 : 0));
}
// Index of (a, b), a <= b, in the packed upper triangle (36 entries).
__host__ __device__ constexpr int tri_index(int a, int b) {
    return a <= b ? a * 8 - a * (a - 1) / 2 + (b - a) : b * 8 - b * (b - 1) / 2 + (a - b);
}

// Reference-cell derivative of the trilinear shape function of corner a in
// direction j at the Gauss point (q & 1, (q >> 1) & 1, q >> 2), points +-1/sqrt(3).
__host__ __device__ constexpr double ref_grad(int q, int a, int j) {
    constexpr double g = 0.57735026918962576451;  // 1/sqrt(3)
    const double pt[3] = {(q & 1) ? g : -g, ((q >> 1) & 1) ? g : -g, (q >> 2) ? g : -g};
    const double sgn[3] = {corner_x(a) ? 1.0 : -1.0, corner_y(a) ? 1.0 : -1.0,
                           corner_z(a) ? 1.0 : -1.0};
    double v = 0.125;
    for (int i = 0; i < 3; ++i) v *= (i == j) ? sgn[i] : (1.0 + sgn[i] * pt[i]);
    return v;
}

struct RefGradTable {
    double v[8][8][3];  // [Gauss point][corner][direction]
};
__host__ __device__ constexpr RefGradTable make_ref_grad_table() {
    RefGradTable t{};
    for (int q = 0; q < 8; ++q)
        for (int a = 0; a < 8; ++a)
            for (int j = 0; j < 3; ++j) t.v[q][a][j] = ref_grad(q, a, j);
    return t;
}
__constant__ RefGradTable kRefGrad = make_ref_grad_table();

// The Jacobian from edge vectors: d x / d xi_j is a weighted sum of the four
// element edges along axis j, E_jk = X(corner with o_j = 1) - X(o_j = 0), with
// weight (1 +- p_a1)(1 +- p_a2) / 8 from the Gauss point's other two
// coordinates (k = c1 + 2 c2 picks the edge by its other-axis corner bits).
struct EdgeWeightTable {
    double w[8][3][4];  // [Gauss point][axis j][edge k]
};
__host__ __device__ constexpr EdgeWeightTable make_edge_weight_table() {
    EdgeWeightTable t{};
    constexpr double g = 0.57735026918962576451;  // 1/sqrt(3)
    for (int q = 0; q < 8; ++q) {
        const double pt[3] = {(q & 1) ? g : -g, ((q >> 1) & 1) ? g : -g, (q >> 2) ? g : -g};
        for (int j = 0; j < 3; ++j) {
            const int a1 = j == 0 ? 1 : 0, a2 = j == 2 ? 1 : 2;
            for (int k = 0; k < 4; ++k) {
                const double s1 = (k & 1) ? 1.0 : -1.0, s2 = (k >> 1) ? 1.0 : -1.0;
                t.w[q][j][k] = 0.125 * (1.0 + s1 * pt[a1]) * (1.0 + s2 * pt[a2]);
            }
        }
    }
    return t;
}
__constant__ EdgeWeightTable kEdgeW = make_edge_weight_table();

// corner of the edge k along axis j at end e (0 or 1)
__host__ __device__ constexpr int edge_corner(int j, int k, int e) {
    const int c1 = k & 1, c2 = k >> 1;
    return j == 0 ? corner_of(e, c1, c2) : (j == 1 ? corner_of(c1, e, c2) : corner_of(c1, c2, e));
}

// For an element whose four edges along each axis are equal (a
// parallelepiped: the trilinear map is affine and its Jacobian constant), the
// quadrature sum K_ab = sum_q grad N_a(q) . grad N_b(q) det J factors as
// K_ab = sum_{j,l} C_jl S^{jl}_ab with the constant metric C = det J J^-1 J^-T
// and S^{jl}_ab = sum_q d_j N_a(q) d_l N_b(q), the same reference-gradient
// products summed over the eight points ahead of time.  Six symmetric pairs
// (j,l) = (0,0) (1,1) (2,2) (0,1) (0,2) (1,2); an off-diagonal pair holds
// both orders, since C_jl = C_lj.
struct AffineTable {
    double s[6][36];  // [pair][packed upper-triangle entry]
};
__host__ __device__ constexpr AffineTable make_affine_table() {
    AffineTable t{};
    constexpr int pj[6] = {0, 1, 2, 0, 0, 1}, pl[6] = {0, 1, 2, 1, 2, 2};
    for (int p = 0; p < 6; ++p)
        for (int a = 0; a < 8; ++a)
            for (int b = a; b < 8; ++b) {
                double v = 0.0;
                for (int q = 0; q < 8; ++q) {
                    v += ref_grad(q, a, pj[p]) * ref_grad(q, b, pl[p]);
                    if (pj[p] != pl[p]) v += ref_grad(q, a, pl[p]) * ref_grad(q, b, pj[p]);
                }
                t.s[p][tri_index(a, b)] = v;
            }
    return t;
}
__constant__ AffineTable kAffine = make_affine_table();

// J^-1 (as the transposed cofactor matrix over det) and det J
__device__ __forceinline__ double jac_inverse(const double J[3][3], double Ji[3][3]) {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double rdet = 1.0 / det;
    Ji[0][0] = c00 * rdet;
    Ji[1][0] = c01 * rdet;
    Ji[2][0] = c02 * rdet;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * rdet;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * rdet;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * rdet;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * rdet;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * rdet;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * rdet;
    return det;
}

// PARALLELEPIPEDS = true: the elements whose edges along each axis agree
// (constant Jacobian); false: all others, by per-point quadrature.  Two
// launches, so that the common constant-Jacobian case does not carry the
// quadrature's registers (224) and runs at full occupancy.
template <bool PARALLELEPIPEDS>
__global__ void __launch_bounds__(128, PARALLELEPIPEDS ? 4 : 1)
k_element_matrices(int nx, int ny, int nz, const double *__restrict__ coords,
                   double *__restrict__ work) {
    const int64_t ne = (int64_t)nx * ny * nz;
    const int64_t nxn = nx + 1, plane = nxn * (ny + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ex = (int)(e % nx);
        const int64_t q0 = e / nx;
        const int ey = (int)(q0 % ny);
        const int ez = (int)(q0 / ny);
        const int64_t n0 = ex + nxn * (ey + (int64_t)(ny + 1) * ez);
        // corner offsets from corner 0: the operator is translation invariant,
        // and offsets of size h keep the Jacobian free of cancellation
        double X[8][3];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int64_t node = n0 + corner_x(a) + nxn * corner_y(a) + plane * corner_z(a);
#pragma unroll
            for (int i = 0; i < 3; ++i) X[a][i] = coords[3 * node + i];
        }
        // axis-aligned brick: a corner's x depends only on its x bit, y on its
        // y bit, z on its z bit, bit for bit (integer compares, no FP64 work)
        bool brick = true;
#pragma unroll
        for (int a = 1; a < 8; ++a) {
            brick = brick && __double_as_longlong(X[a][0]) == __double_as_longlong(X[corner_of(corner_x(a), 0, 0)][0]);
            brick = brick && __double_as_longlong(X[a][1]) == __double_as_longlong(X[corner_of(0, corner_y(a), 0)][1]);
            brick = brick && __double_as_longlong(X[a][2]) == __double_as_longlong(X[corner_of(0, 0, corner_z(a))][2]);
        }
        if (brick) {
            if constexpr (!PARALLELEPIPEDS) continue;   // the parallelepiped launch's element
            // the parallelepiped path below with J = diag(hx, hy, hz) / 2: the
            // same operations less the ones on exact zeros (bit-identical)
            const double J0 = 0.5 * (X[1][0] - X[0][0]);
            const double J1 = 0.5 * (X[3][1] - X[0][1]);
            const double J2 = 0.5 * (X[4][2] - X[0][2]);
            const double c00 = J1 * J2;
            const double det = J0 * c00;
            const double rdet = 1.0 / det;
            const double i0 = c00 * rdet, i1 = (J0 * J2) * rdet, i2 = (J0 * J1) * rdet;
            const double C0 = det * (i0 * i0), C1 = det * (i1 * i1), C2 = det * (i2 * i2);
            double *w = work + e;   // entry k at w[k ne]
#pragma unroll 4
            for (int k = 0; k < 36; ++k, w += ne) {
                double v = C0 * kAffine.s[0][k];
                v = fma(C1, kAffine.s[1][k], v);
                *w = fma(C2, kAffine.s[2][k], v);
            }
            continue;
        }
#pragma unroll
        for (int a = 7; a >= 0; --a)
#pragma unroll
            for (int i = 0; i < 3; ++i) X[a][i] -= X[0][i];
        if constexpr (PARALLELEPIPEDS) {
            // parallelepiped: the four edges along each axis agree bit for bit;
            // then d x_i / d xi_j = E_j / 2 is constant (reference cell [-1, 1]^3)
            bool affine = true;
            double J[3][3], Ji[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double e0 = X[edge_corner(j, 0, 1)][i] - X[edge_corner(j, 0, 0)][i];
#pragma unroll
                    for (int k = 1; k < 4; ++k) {
                        const double ek = X[edge_corner(j, k, 1)][i] - X[edge_corner(j, k, 0)][i];
                        affine = affine && __double_as_longlong(ek) == __double_as_longlong(e0);
                    }
                    J[i][j] = 0.5 * e0;
                }
            if (!affine) continue;   // the quadrature launch's element
            const double det = jac_inverse(J, Ji);
            // C_jl = det sum_i Ji[j][i] Ji[l][i], pairs in the table's order
            constexpr int pj[6] = {0, 1, 2, 0, 0, 1}, pl[6] = {0, 1, 2, 1, 2, 2};
            double C[6];
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                double c = Ji[pj[p]][0] * Ji[pl[p]][0];
                c = fma(Ji[pj[p]][1], Ji[pl[p]][1], c);
                c = fma(Ji[pj[p]][2], Ji[pl[p]][2], c);
                C[p] = det * c;
            }
            double *w = work + e;   // entry k at w[k ne]
#pragma unroll 4
            for (int k = 0; k < 36; ++k, w += ne) {
                double v = C[0] * kAffine.s[0][k];
#pragma unroll
                for (int p = 1; p < 6; ++p) v = fma(C[p], kAffine.s[p][k], v);
                *w = v;
            }
            continue;
        } else {
            // the twelve edge vectors (once per element)
            double E[3][4][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int i = 0; i < 3; ++i) E[j][k][i] = X[edge_corner(j, k, 1)][i] - X[edge_corner(j, k, 0)][i];
            bool affine = true;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 1; k < 4; ++k)
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        affine = affine && __double_as_longlong(E[j][k][i]) == __double_as_longlong(E[j][0][i]);
            if (affine) continue;   // the parallelepiped launch's element
            double K[36];
#pragma unroll
            for (int k = 0; k < 36; ++k) K[k] = 0.0;

#pragma unroll 1
            for (int q = 0; q < 8; ++q) {
                // J[i][j] = d x_i / d xi_j = sum over the four edges along j
                double J[3][3];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        double s = 0.0;
#pragma unroll
                        for (int k = 0; k < 4; ++k) s = fma(E[j][k][i], kEdgeW.w[q][j][k], s);
                        J[i][j] = s;
                    }
                double Ji[3][3];
                const double det = jac_inverse(J, Ji);
                // physical gradients G[a] = J^{-T} grad_xi N_a; weight 1 at every point
                double G[8][3];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        double s = 0.0;
#pragma unroll
                        for (int j = 0; j < 3; ++j) s = fma(Ji[j][i], kRefGrad.v[q][a][j], s);
                        G[a][i] = s;
                    }
                double H[8][3];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int i = 0; i < 3; ++i) H[a][i] = det * G[a][i];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = a; b < 8; ++b) {
                        double d = H[a][0] * G[b][0];
                        d = fma(H[a][1], G[b][1], d);
                        d = fma(H[a][2], G[b][2], d);
                        K[tri_index(a, b)] += d;
                    }
            }
#pragma unroll
            for (int k = 0; k < 36; ++k) work[k * ne + e] = K[k];
        }
    }
}

// Closed-form CSR row start of node (ix, iy, iz): the prefix sum, in node
// order, of the per-row neighbour counts cx(ix) cy(iy) cz(iz).
__device__ __forceinline__ int64_t axis_count(int i, int n) {  // n = elements on the axis
    return (i == 0 || i == n) ? 2 : 3;
}
__device__ __forceinline__ int64_t axis_prefix(int i) {  // sum of counts of indices < i
    return i == 0 ? 0 : 3 * (int64_t)i - 1;
}

// One warp per 32 consecutive rows (contiguous in CSR): each lane gathers its
// row from the element workspace (the up to 64 loads issued without branches,
// zeros for missing elements), writes the row into the warp's shared-memory
// slice at its exclusive-scan offset, and the warp stores the slice with
// coalesced writes.
constexpr int kAsmWarps = 4;
constexpr int kAsmSlice = 32 * 27;   // entries of 32 full rows

__global__ void __launch_bounds__(32 * kAsmWarps)
k_assemble_rows(int nx, int ny, int nz, const double *__restrict__ work,
                const uint8_t *__restrict__ bc_flag, const double *__restrict__ bc_val,
                int32_t *__restrict__ row_ptr, int32_t *__restrict__ cols,
                double *__restrict__ vals, double *__restrict__ b) {
    __shared__ int32_t s_cols[kAsmWarps][kAsmSlice];
    __shared__ double s_vals[kAsmWarps][kAsmSlice];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nxn = nx + 1, nyn = ny + 1;
    const int64_t m = nxn * nyn * (nz + 1);
    const int64_t ne = (int64_t)nx * ny * nz;
    const int64_t Cx = 3 * (int64_t)nx + 1, Cy = 3 * (int64_t)ny + 1;
    const int64_t ngroups = (m + 31) / 32;
    for (int64_t grp = (int64_t)blockIdx.x * kAsmWarps + wib; grp < ngroups;
         grp += (int64_t)gridDim.x * kAsmWarps) {
        const int64_t i = grp * 32 + lane;
        const bool live = i < m;
        const int64_t ii = live ? i : m - 1;
        const int ix = (int)(ii % nxn);
        const int64_t q = ii / nxn;
        const int iy = (int)(q % nyn);
        const int iz = (int)(q / nyn);

        double acc[27];
#pragma unroll
        for (int k = 0; k < 27; ++k) acc[k] = 0.0;
        // incident elements (ix+dx, iy+dy, iz+dz), dx,dy,dz in {-1,0}, in element-id order
#pragma unroll
        for (int dz = -1; dz <= 0; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 0; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 0; ++dx) {
                    const int ex = ix + dx, ey = iy + dy, ez = iz + dz;
                    const bool has = ex >= 0 && ex < nx && ey >= 0 && ey < ny && ez >= 0 && ez < nz;
                    const int64_t e = has ? ex + (int64_t)nx * (ey + (int64_t)ny * ez) : 0;
                    const int a = corner_of(-dx, -dy, -dz);
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) {
                        const int sx = dx + corner_x(bb), sy = dy + corner_y(bb), sz = dz + corner_z(bb);
                        const int slot = (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
                        acc[slot] += has ? work[(int64_t)tri_index(a, bb) * ne + e] : 0.0;
                    }
                }

        const int64_t start = Cx * Cy * axis_prefix(iz) + Cx * axis_count(iz, nz) * axis_prefix(iy) +
                              axis_count(iy, ny) * axis_count(iz, nz) * axis_prefix(ix);
        const int cnt = live ? (int)(axis_count(ix, nx) * axis_count(iy, ny) * axis_count(iz, nz)) : 0;
        if (live) row_ptr[i] = (int32_t)start;
        if (i == m - 1) row_ptr[m] = (int32_t)(start + cnt);
        // exclusive scan of the row lengths: the row's place in the warp's slice
        int off = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, off, d);
            if (lane >= d) off += t;
        }
        const int total = __shfl_sync(0xffffffffu, off, 31);
        off -= cnt;
        const int64_t start0 = __shfl_sync(0xffffffffu, start, 0);

        const bool brow = live && bc_flag[ii] != 0;
        double bi = 0.0;
        int pos = off;
        if (live) {
#pragma unroll
            for (int sz = -1; sz <= 1; ++sz)
#pragma unroll
                for (int sy = -1; sy <= 1; ++sy)
#pragma unroll
                    for (int sx = -1; sx <= 1; ++sx) {
                        const int jx = ix + sx, jy = iy + sy, jz = iz + sz;
                        if (jx < 0 || jx > nx || jy < 0 || jy > ny || jz < 0 || jz > nz) continue;
                        const int64_t j = i + sx + nxn * (sy + nyn * sz);
                        double v = acc[(sz + 1) * 9 + (sy + 1) * 3 + (sx + 1)];
                        if (brow) {
                            v = (j == i) ? 1.0 : 0.0;
                        } else if (bc_flag[j]) {
                            bi = fma(-v, bc_val[j], bi);
                            v = 0.0;
                        }
                        s_cols[wib][pos] = (int32_t)j;
                        s_vals[wib][pos] = v;
                        ++pos;
                    }
            b[i] = brow ? bc_val[i] : bi;
        }
        __syncwarp();
        for (int t = lane; t < total; t += 32) {
            cols[start0 + t] = s_cols[wib][t];
            vals[start0 + t] = s_vals[wib][t];
        }
        __syncwarp();
    }
}

static int grid_cap(int64_t n, int threads, int per_sm) {
    int64_t blocks = (n + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (cap < 1) cap = 1024;
    return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_assemble_workspace(int nx, int ny, int nz, size_t *h_bytes) {
    fe_sizes sz;
    fe_status st = fe_problem_sizes(nx, ny, nz, &sz);
    if (st != FE_OK) return st;
    if (h_bytes == nullptr) return FE_ERR_ARG;
    *h_bytes = (size_t)sz.n_elems * 36 * sizeof(double);
    return FE_OK;
}

fe_status fe_assemble_csr(int nx, int ny, int nz, const double *d_coords,
                          const uint8_t *d_bc_flag, const double *d_bc_val, int32_t *d_row_ptr,
                          int32_t *d_cols, double *d_vals, double *d_b, void *d_work,
                          size_t work_bytes, fe_stream_t stream) {
    fe_sizes sz;
    fe_status st = fe_problem_sizes(nx, ny, nz, &sz);
    if (st != FE_OK) return st;
    if (!d_coords || !d_bc_flag || !d_bc_val || !d_row_ptr || !d_cols || !d_vals || !d_b || !d_work)
        return FE_ERR_ARG;
    if (!aligned(d_coords, 8) || !aligned(d_bc_val, 8) || !aligned(d_vals, 8) || !aligned(d_b, 8) ||
        !aligned(d_work, 8) || !aligned(d_row_ptr, 4) || !aligned(d_cols, 4))
        return FE_ERR_ARG;
    if (work_bytes < (size_t)sz.n_elems * 36 * sizeof(double)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    k_element_matrices<true><<<grid_cap(sz.n_elems, 128, 32), 128, 0, s>>>(nx, ny, nz, d_coords,
                                                                           (double *)d_work);
    FE_TRY_LAUNCH();
    k_element_matrices<false><<<grid_cap(sz.n_elems, 128, 32), 128, 0, s>>>(nx, ny, nz, d_coords,
                                                                            (double *)d_work);
    FE_TRY_LAUNCH();
    k_assemble_rows<<<grid_cap((sz.n_rows + 31) / 32, kAsmWarps, 32), 32 * kAsmWarps, 0, s>>>(
        nx, ny, nz, (const double *)d_work, d_bc_flag, d_bc_val, d_row_ptr, d_cols, d_vals, d_b);
    FE_TRY_LAUNCH();
    return FE_OK;
}

}  // extern "C"
