/*
 * fe_oracle.c -- plain, serial FP64 CPU oracle for the MiniFE heat-conduction
 * path studied in "The Research and Optimization of Parallel Finite Element
 * Algorithm based on MiniFE" (arXiv 1505.08023).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the GPU library never does, and the two
 * share no source, header, table or helper.  Every routine is written to be
 * checked by eye against the paper, not to be fast:
 *
 *   mesh processing        paper Sec. 1 (problem statement, mesh module)
 *   matrix generation      paper Sec. 1 and Fig 3.6 (neighbour count -> CRS)
 *   element operator       paper Sec. 1 ("element operator computing")
 *   FE assembly            paper Sec. 1 and Fig 3.7 (element loop + scatter)
 *   Dirichlet rows         paper Sec. 1 (boundary rows recorded by the mesh)
 *   CRS SpMV               paper Fig 3.1
 *   BCRS conversion/SpMV   paper Sec. 3.1, Fig 3.2
 *   CG                     paper Sec. 1 (WAXPY, DOT, MATVEC; no preconditioner)
 *
 * Readings of points the paper leaves open (node numbering, per-axis neighbour
 * bounds, symmetric Dirichlet elimination, zero source term, stopping rule on
 * ||r||/||b||) are stated at each routine.  Build with -ffp-contract=off so
 * that every operation is one IEEE FP64 rounding on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Mesh (paper Sec. 1: unit cube 0<=x,y,z<=1, Nx x Ny x Nz hexahedra).       */
/* Reading: node id = ix + (nx+1)*(iy + (ny+1)*iz), x fastest.               */
/* ------------------------------------------------------------------------ */

static int64_t node_id(int nx, int ny, int ix, int iy, int iz)
{
    return (int64_t)ix + (int64_t)(nx + 1) * ((int64_t)iy + (int64_t)(ny + 1) * iz);
}

int64_t orc_num_nodes(int nx, int ny, int nz)
{
    return (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
}

/*
 * Node coordinates, boundary flag and prescribed value.
 *
 * face_vals == NULL: the paper's problem -- T = 1 on the plane x = 1 (the
 * whole closed plane, edges and corners included), T = 0 on the other faces.
 *
 * face_vals != NULL: one value per boundary-face node, faces concatenated in
 * the order x0, x1, y0, y1, z0, z1; an x face is indexed iy + (ny+1)*iz, a y
 * face ix + (nx+1)*iz, a z face ix + (nx+1)*iy.  Faces are applied in that
 * order, so a later face overwrites an earlier one on a shared edge.
 */
void orc_mesh(int nx, int ny, int nz, const double *face_vals,
              double *coords, uint8_t *bc_flag, double *bc_val)
{
    for (int iz = 0; iz <= nz; ++iz)
        for (int iy = 0; iy <= ny; ++iy)
            for (int ix = 0; ix <= nx; ++ix) {
                int64_t i = node_id(nx, ny, ix, iy, iz);
                coords[3 * i + 0] = (double)ix / (double)nx;
                coords[3 * i + 1] = (double)iy / (double)ny;
                coords[3 * i + 2] = (double)iz / (double)nz;
                int on_boundary = (ix == 0 || ix == nx || iy == 0 || iy == ny ||
                                   iz == 0 || iz == nz);
                bc_flag[i] = (uint8_t)on_boundary;
                bc_val[i] = 0.0;
                if (face_vals == NULL) {
                    if (ix == nx)
                        bc_val[i] = 1.0;
                    continue;
                }
                int64_t sx = (int64_t)(ny + 1) * (nz + 1);
                int64_t sy = (int64_t)(nx + 1) * (nz + 1);
                int64_t base_x1 = sx, base_y0 = 2 * sx, base_y1 = 2 * sx + sy;
                int64_t base_z0 = 2 * sx + 2 * sy;
                int64_t base_z1 = base_z0 + (int64_t)(nx + 1) * (ny + 1);
                if (ix == 0)  bc_val[i] = face_vals[iy + (int64_t)(ny + 1) * iz];
                if (ix == nx) bc_val[i] = face_vals[base_x1 + iy + (int64_t)(ny + 1) * iz];
                if (iy == 0)  bc_val[i] = face_vals[base_y0 + ix + (int64_t)(nx + 1) * iz];
                if (iy == ny) bc_val[i] = face_vals[base_y1 + ix + (int64_t)(nx + 1) * iz];
                if (iz == 0)  bc_val[i] = face_vals[base_z0 + ix + (int64_t)(nx + 1) * iy];
                if (iz == nz) bc_val[i] = face_vals[base_z1 + ix + (int64_t)(nx + 1) * iy];
            }
}

/* Local hex8 node order: (0,0,0),(1,0,0),(1,1,0),(0,1,0),(0,0,1),(1,0,1),(1,1,1),(0,1,1). */
static const int HEX8_CORNER[8][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
    {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

/* Element id e = ex + nx*(ey + ny*ez); its eight global node ids. */
void orc_element_nodes(int nx, int ny, int nz, int64_t e, int64_t nodes[8])
{
    (void)nz;
    int ex = (int)(e % nx);
    int ey = (int)((e / nx) % ny);
    int ez = (int)(e / ((int64_t)nx * ny));
    for (int a = 0; a < 8; ++a)
        nodes[a] = node_id(nx, ny, ex + HEX8_CORNER[a][0], ey + HEX8_CORNER[a][1],
                           ez + HEX8_CORNER[a][2]);
}

/* ------------------------------------------------------------------------ */
/* Element operator (paper Sec. 1): K_ab = integral grad N_a . grad N_b over */
/* the hexahedron, trilinear shape functions, 2x2x2 Gauss-Legendre rule      */
/* (points +-1/sqrt(3), weights 1), Jacobian taken from the node coords.     */
/* X[3*a + i] = coordinate i of local node a; K is row-major 8x8.            */
/* The operator depends on the element's shape only, so the Jacobian is      */
/* built from corner offsets X_a - X_0: the same integral without the        */
/* cancellation of summing absolute coordinates of size 1 into entries of    */
/* size h.                                                                   */
/* ------------------------------------------------------------------------ */
void orc_element_matrix(const double *Xabs, double *K)
{
    double X[24];
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i)
            X[3 * a + i] = Xabs[3 * a + i] - Xabs[i];

    const double g = 1.0 / sqrt(3.0);
    const double gauss_pt[2] = {-g, g};
    for (int k = 0; k < 64; ++k)
        K[k] = 0.0;

    for (int qz = 0; qz < 2; ++qz)
        for (int qy = 0; qy < 2; ++qy)
            for (int qx = 0; qx < 2; ++qx) {
                double xi = gauss_pt[qx], eta = gauss_pt[qy], zeta = gauss_pt[qz];
                double weight = 1.0;

                /* derivatives of N_a = (1+s xi)(1+t eta)(1+u zeta)/8 in reference coords */
                double dN[8][3];
                for (int a = 0; a < 8; ++a) {
                    double s = 2.0 * HEX8_CORNER[a][0] - 1.0;
                    double t = 2.0 * HEX8_CORNER[a][1] - 1.0;
                    double u = 2.0 * HEX8_CORNER[a][2] - 1.0;
                    dN[a][0] = 0.125 * s * (1.0 + t * eta) * (1.0 + u * zeta);
                    dN[a][1] = 0.125 * (1.0 + s * xi) * t * (1.0 + u * zeta);
                    dN[a][2] = 0.125 * (1.0 + s * xi) * (1.0 + t * eta) * u;
                }

                /* J[i][j] = d x_i / d xi_j */
                double J[3][3] = {{0}};
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        for (int a = 0; a < 8; ++a)
                            J[i][j] += X[3 * a + i] * dN[a][j];

                double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                           - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                           + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);

                /* inverse by cofactors: Jinv[i][j] = cof(J)[j][i] / det */
                double Jinv[3][3];
                Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
                Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
                Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
                Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;

                /* physical gradients: grad_x N_a = J^{-T} grad_xi N_a */
                double G[8][3];
                for (int a = 0; a < 8; ++a)
                    for (int i = 0; i < 3; ++i) {
                        G[a][i] = 0.0;
                        for (int j = 0; j < 3; ++j)
                            G[a][i] += Jinv[j][i] * dN[a][j];
                    }

                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b) {
                        double d = G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2];
                        K[8 * a + b] += weight * det * d;
                    }
            }
}

/* ------------------------------------------------------------------------ */
/* Matrix generation (paper Sec. 1, Fig 3.6): for every node count the       */
/* 3x3x3 neighbours that exist, prefix-sum into the CRS row pointer, then    */
/* list the neighbour ids.  Reading: the existence test is per axis          */
/* (0 <= ix+sx <= nx, likewise y and z), which gives (3n-2)^3 entries on a   */
/* cube with n nodes per axis.  Columns come out ascending because sz, sy,   */
/* sx run from -1 to 1 with x fastest in the node id.                        */
/* Returns nnz, or -1 if nnz does not fit an int32 row pointer.  With        */
/* row_ptr == NULL only the count is returned.                               */
/* ------------------------------------------------------------------------ */
int64_t orc_pattern(int nx, int ny, int nz, int32_t *row_ptr, int32_t *cols)
{
    int64_t m = orc_num_nodes(nx, ny, nz);
    int64_t nnz = 0;
    for (int64_t i = 0; i < m; ++i) {
        int ix = (int)(i % (nx + 1));
        int iy = (int)((i / (nx + 1)) % (ny + 1));
        int iz = (int)(i / ((int64_t)(nx + 1) * (ny + 1)));
        int count = 0;
        for (int sz = -1; sz <= 1; ++sz)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    int jx = ix + sx, jy = iy + sy, jz = iz + sz;
                    if (jx >= 0 && jx <= nx && jy >= 0 && jy <= ny && jz >= 0 && jz <= nz)
                        ++count;
                }
        if (row_ptr != NULL)
            row_ptr[i] = (int32_t)nnz;
        nnz += count;
        if (nnz > INT32_MAX)
            return -1;
    }
    if (row_ptr == NULL)
        return nnz;
    row_ptr[m] = (int32_t)nnz;

    for (int64_t i = 0; i < m; ++i) {
        int ix = (int)(i % (nx + 1));
        int iy = (int)((i / (nx + 1)) % (ny + 1));
        int iz = (int)(i / ((int64_t)(nx + 1) * (ny + 1)));
        int64_t pos = row_ptr[i];
        for (int sz = -1; sz <= 1; ++sz)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    int jx = ix + sx, jy = iy + sy, jz = iz + sz;
                    if (jx >= 0 && jx <= nx && jy >= 0 && jy <= ny && jz >= 0 && jz <= nz)
                        cols[pos++] = (int32_t)node_id(nx, ny, jx, jy, jz);
                }
    }
    return nnz;
}

/* Position of column c in row i of a CRS matrix with sorted columns, or -1. */
static int64_t find_in_row(const int32_t *row_ptr, const int32_t *cols, int64_t i, int64_t c)
{
    int64_t lo = row_ptr[i], hi = row_ptr[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cols[mid] == c)
            return mid;
        if (cols[mid] < c)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* FE assembly (paper Sec. 1 and Fig 3.7), serial: for every element in id   */
/* order, gather its nodes and coordinates, compute the element matrix and   */
/* add it into the global CRS values.  Reading: steady conduction with no    */
/* source, so the element vector is zero and b receives nothing here.        */
/* vals and b are overwritten.  Returns 0, or -1 if a column is missing.     */
/* ------------------------------------------------------------------------ */
int orc_assemble(int nx, int ny, int nz, const double *coords,
                 const int32_t *row_ptr, const int32_t *cols, double *vals, double *b)
{
    int64_t m = orc_num_nodes(nx, ny, nz);
    int64_t ne = (int64_t)nx * ny * nz;
    for (int64_t k = 0; k < row_ptr[m]; ++k)
        vals[k] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        b[i] = 0.0;

    for (int64_t e = 0; e < ne; ++e) {
        int64_t nodes[8];
        double X[24], K[64];
        orc_element_nodes(nx, ny, nz, e, nodes);
        for (int a = 0; a < 8; ++a)
            for (int i = 0; i < 3; ++i)
                X[3 * a + i] = coords[3 * nodes[a] + i];
        orc_element_matrix(X, K);
        for (int a = 0; a < 8; ++a)
            for (int bb = 0; bb < 8; ++bb) {
                int64_t pos = find_in_row(row_ptr, cols, nodes[a], nodes[bb]);
                if (pos < 0)
                    return -1;
                vals[pos] += K[8 * a + bb];
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Dirichlet conditions on the rows the mesh module recorded (paper Sec. 1). */
/* Reading: symmetric elimination, which keeps A symmetric positive definite */
/* for CG.  A boundary row becomes the identity row (diagonal 1, stored      */
/* off-diagonals 0) with b_i = g_i; in every other row each boundary column  */
/* j moves to the right-hand side, b_i -= a_ij g_j, and a_ij becomes 0.  The */
/* sparsity pattern does not change.                                         */
/* ------------------------------------------------------------------------ */
void orc_dirichlet(int64_t m, const uint8_t *bc_flag, const double *bc_val,
                   const int32_t *row_ptr, const int32_t *cols, double *vals, double *b)
{
    for (int64_t i = 0; i < m; ++i) {
        if (bc_flag[i]) {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                vals[k] = (cols[k] == i) ? 1.0 : 0.0;
            b[i] = bc_val[i];
        } else {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                if (bc_flag[cols[k]]) {
                    b[i] -= vals[k] * bc_val[cols[k]];
                    vals[k] = 0.0;
                }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* CRS SpMV, y = A x (paper Fig 3.1).  By the definition of the CRS format, */
/* row i stores the pairs (cols[k], vals[k]) for row_ptr[i] <= k <           */
/* row_ptr[i+1], so y_i is the inner product of those values with the x      */
/* entries they name, summed in stored (ascending column) order.             */
/* ------------------------------------------------------------------------ */
static double crs_row_product(const int32_t *row_ptr, const int32_t *cols, const double *vals,
                              const double *x, int64_t i)
{
    const int64_t first = row_ptr[i], count = (int64_t)row_ptr[i + 1] - first;
    double s = 0.0;
    for (int64_t t = 0; t < count; ++t)
        s += vals[first + t] * x[cols[first + t]];
    return s;
}

void orc_spmv_csr(int64_t m, const int32_t *row_ptr, const int32_t *cols,
                  const double *vals, const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i)
        y[i] = crs_row_product(row_ptr, cols, vals, x, i);
}

/* ------------------------------------------------------------------------ */
/* The paper's BCRS with 1 x n segments of variable length (Sec. 3.1):       */
/* a segment is a maximal run of adjacent columns in a row; jas holds each   */
/* segment's first column, offsets each segment's first value, ptr each      */
/* row's first segment.  val is the CRS value array unchanged.               */
/* With jas == NULL only nns is returned.                                    */
/* ------------------------------------------------------------------------ */
int64_t orc_csr_to_bcrs(int64_t m, const int32_t *row_ptr, const int32_t *cols,
                        int32_t *jas, int32_t *offsets, int32_t *ptr)
{
    int64_t nns = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (ptr != NULL)
            ptr[i] = (int32_t)nns;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int starts_segment = (k == row_ptr[i]) || (cols[k] != cols[k - 1] + 1);
            if (starts_segment) {
                if (jas != NULL) {
                    jas[nns] = cols[k];
                    offsets[nns] = (int32_t)k;
                }
                ++nns;
            }
        }
    }
    if (ptr != NULL) {
        ptr[m] = (int32_t)nns;
        offsets[nns] = row_ptr[m];
    }
    return nns;
}

/* BCRS SpMV (paper Sec. 3.1, Fig 3.2).  By the format's definition segment */
/* j of row i (ptr[i] <= j < ptr[i+1]) is the run of L_j = offsets[j+1] -    */
/* offsets[j] adjacent columns jas[j], jas[j]+1, ..., whose values are       */
/* val[offsets[j] + t], t < L_j; y_i sums value times x over the segments in */
/* order, which is the CRS order of the same entries.                        */
void orc_spmv_bcrs(int64_t m, const int32_t *ptr, const int32_t *jas,
                   const int32_t *offsets, const double *val, const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = ptr[i]; j < ptr[i + 1]; ++j) {
            const double *seg_val = val + offsets[j];
            const double *seg_x = x + jas[j];
            const int64_t len = (int64_t)offsets[j + 1] - offsets[j];
            for (int64_t t = 0; t < len; ++t)
                s += seg_val[t] * seg_x[t];
        }
        y[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Vector kernels named in the paper's CG module (Sec. 1): DOT and WAXPY.    */
/* Reading of DOT: the inner product of the two vectors, rounded once.  A    */
/* plain running sum in index order carries a rounding error that grows      */
/* with n (up to n u relative) and, through CG's sensitivity to its          */
/* inner products, moves the stop step of a 10^6-row solve by several steps  */
/* away from every accurately summed order.  So DOT is the compensated dot   */
/* product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product",    */
/* SIAM J. Sci. Comput. 26, 2005): each product split exactly into p + e     */
/* (Dekker's product with Veltkamp's splitting), the running sum kept with   */
/* its exact rounding error (Knuth's TwoSum), the errors summed on the side  */
/* and added once at the end.  The result is as accurate as the inner        */
/* product computed in twice the working precision and then rounded:         */
/* |DOT - a.b| <= u |a.b| + gamma_n^2 |a|.|b|.  Plain operations only, in    */
/* index order, so x86 and Arm give the same bits.                           */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double *s, double *err)
{
    const double x = a + b, z = x - a;
    *s = x;
    *err = (a - (x - z)) + (b - z);
}

static void veltkamp_split(double a, double *hi, double *lo)
{
    const double c = 134217729.0 * a;         /* (2^27 + 1) a */
    const double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}

static void two_product(double a, double b, double *p, double *err)
{
    double ah, al, bh, bl;
    const double x = a * b;
    veltkamp_split(a, &ah, &al);
    veltkamp_split(b, &bh, &bl);
    *p = x;
    *err = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
}

double orc_dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double p, ep, q;
        two_product(a[i], b[i], &p, &ep);
        two_sum(s, p, &s, &q);
        c += q + ep;
    }
    return s + c;
}

/* w = alpha x + beta y */
void orc_waxpby(int64_t n, double alpha, const double *x, double beta, const double *y, double *w)
{
    for (int64_t i = 0; i < n; ++i)
        w[i] = alpha * x[i] + beta * y[i];
}

/* ------------------------------------------------------------------------ */
/* Unpreconditioned CG (paper Sec. 1: MATVEC, DOT, WAXPY), textbook form:    */
/*   r = b - A x, p = r                                                      */
/*   repeat: w = A p; alpha = r.r / p.w; x += alpha p; r -= alpha w;         */
/*           beta = r'.r' / r.r; p = r' + beta p                             */
/* Reading of the stopping rule: stop once ||r_k|| <= tol ||b|| (recursive   */
/* residual, checked before the first step and after every update) or after  */
/* maxit steps.  b = 0 gives x = 0 at once.                                  */
/* Returns 0 converged, 1 hit maxit, 2 breakdown (p.w <= 0 or not finite).   */
/* x holds the start vector on entry and the iterate on exit.                */
/* ------------------------------------------------------------------------ */
int orc_cg(int64_t m, const int32_t *row_ptr, const int32_t *cols, const double *vals,
           const double *b, double *x, double tol, int maxit,
           int *iters_out, double *relres_out)
{
    double *r = (double *)malloc((size_t)m * sizeof(double));
    double *p = (double *)malloc((size_t)m * sizeof(double));
    double *w = (double *)malloc((size_t)m * sizeof(double));
    int status = 1, k = 0;
    double bb = orc_dot(m, b, b);
    double rr = 0.0;

    if (bb == 0.0) {
        for (int64_t i = 0; i < m; ++i)
            x[i] = 0.0;
        status = 0;
        goto done;
    }
    orc_spmv_csr(m, row_ptr, cols, vals, x, w);
    orc_waxpby(m, 1.0, b, -1.0, w, r);              /* r = b - A x */
    for (int64_t i = 0; i < m; ++i)
        p[i] = r[i];
    rr = orc_dot(m, r, r);

    while (1) {
        if (rr <= tol * tol * bb) {
            status = 0;
            break;
        }
        if (k >= maxit) {
            status = 1;
            break;
        }
        orc_spmv_csr(m, row_ptr, cols, vals, p, w);  /* w = A p */
        double pw = orc_dot(m, p, w);
        if (!(pw > 0.0) || !isfinite(pw)) {
            status = 2;
            break;
        }
        double alpha = rr / pw;
        orc_waxpby(m, 1.0, x, alpha, p, x);         /* x = x + alpha p */
        orc_waxpby(m, 1.0, r, -alpha, w, r);        /* r = r - alpha w */
        double rr_new = orc_dot(m, r, r);
        double beta = rr_new / rr;
        rr = rr_new;
        ++k;
        orc_waxpby(m, 1.0, r, beta, p, p);          /* p = r + beta p */
    }
done:
    if (iters_out)
        *iters_out = k;
    if (relres_out)
        *relres_out = (bb == 0.0) ? 0.0 : sqrt(rr / bb);
    free(r);
    free(p);
    free(w);
    return status;
}

/*
 * Single-reduction CG (Chronopoulos and Gear, 1989; the s = 1 member of their
 * s-step family).  In exact arithmetic it produces the iterates of orc_cg.
 * A step performs one product w = A r and forms both inner products it needs,
 * gamma = (r, r) and delta = (w, r), from the same vectors; the curvature
 * p.Ap is not formed directly but follows from
 *     p_k . A p_k = delta_k - beta_k gamma_k / alpha_{k-1}      (k >= 1),
 * and s = A p is carried by the recurrence s_k = w_k + beta_k s_{k-1}.
 * Step k:  beta_k = gamma_k / gamma_{k-1} (beta_0 = 0),
 *          alpha_k = gamma_k / (p_k . A p_k),
 *          p = r + beta p,  s = w + beta s,  x = x + alpha p,  r = r - alpha s,
 *          w = A r,  gamma = (r, r),  delta = (w, r).
 * Stopping rule and status codes as orc_cg (gamma is the recursive r.r).
 * Safeguard: in finite precision the curvature recurrence can lose its sign
 * near convergence (the subtraction cancels); when it gives p.Ap <= 0 (or a
 * non-finite value) the step restarts the direction instead -- beta = 0, so
 * p = r, s = w and p.Ap = delta = r.Ar, positive for an SPD matrix -- and only
 * delta <= 0 is a breakdown.
 */
int orc_cg_sr(int64_t m, const int32_t *row_ptr, const int32_t *cols, const double *vals,
              const double *b, double *x, double tol, int maxit,
              int *iters_out, double *relres_out)
{
    double *r = (double *)malloc((size_t)m * sizeof(double));
    double *w = (double *)malloc((size_t)m * sizeof(double));
    double *p = (double *)calloc((size_t)m, sizeof(double));
    double *s = (double *)calloc((size_t)m, sizeof(double));
    int status = 1, k = 0;
    double bb = orc_dot(m, b, b);
    double gamma = 0.0, gamma_prev = 0.0, delta = 0.0, alpha_prev = 0.0;

    if (bb == 0.0) {
        for (int64_t i = 0; i < m; ++i)
            x[i] = 0.0;
        status = 0;
        goto done;
    }
    orc_spmv_csr(m, row_ptr, cols, vals, x, w);
    orc_waxpby(m, 1.0, b, -1.0, w, r);              /* r = b - A x */
    orc_spmv_csr(m, row_ptr, cols, vals, r, w);     /* w = A r */
    gamma = orc_dot(m, r, r);
    delta = orc_dot(m, w, r);

    while (1) {
        if (gamma <= tol * tol * bb) {
            status = 0;
            break;
        }
        if (k >= maxit) {
            status = 1;
            break;
        }
        double beta = 0.0, curv = delta;
        if (k > 0) {
            beta = gamma / gamma_prev;
            curv = delta - beta * gamma / alpha_prev;
            if (!(curv > 0.0) || !isfinite(curv)) {   /* restart the direction */
                beta = 0.0;
                curv = delta;
            }
        }
        if (!(curv > 0.0) || !isfinite(curv)) {
            status = 2;
            break;
        }
        double alpha = gamma / curv;
        orc_waxpby(m, 1.0, r, beta, p, p);          /* p = r + beta p */
        orc_waxpby(m, 1.0, w, beta, s, s);          /* s = w + beta s */
        orc_waxpby(m, 1.0, x, alpha, p, x);         /* x = x + alpha p */
        orc_waxpby(m, 1.0, r, -alpha, s, r);        /* r = r - alpha s */
        orc_spmv_csr(m, row_ptr, cols, vals, r, w); /* w = A r */
        gamma_prev = gamma;
        gamma = orc_dot(m, r, r);
        delta = orc_dot(m, w, r);
        alpha_prev = alpha;
        ++k;
    }
done:
    if (iters_out)
        *iters_out = k;
    if (relres_out)
        *relres_out = (bb == 0.0) ? 0.0 : sqrt(gamma / bb);
    free(r);
    free(w);
    free(p);
    free(s);
    return status;
}

/* True relative residual ||b - A x|| / ||b|| (0 when b = 0 and A x = 0). */
double orc_true_relres(int64_t m, const int32_t *row_ptr, const int32_t *cols,
                       const double *vals, const double *b, const double *x)
{
    double *ax = (double *)malloc((size_t)m * sizeof(double));
    double *res = (double *)malloc((size_t)m * sizeof(double));
    orc_spmv_csr(m, row_ptr, cols, vals, x, ax);
    orc_waxpby(m, 1.0, b, -1.0, ax, res);
    double rn = orc_dot(m, res, res), bn = orc_dot(m, b, b);
    free(ax);
    free(res);
    if (bn == 0.0)
        return sqrt(rn);
    return sqrt(rn / bn);
}

/* ------------------------------------------------------------------------ */
/* Matrix-free form of the same Dirichlet system (an extension beside the    */
/* paper's stored CRS/BCRS formats: the operator applied without a matrix).  */
/*                                                                          */
/* On the box mesh every element is the same axis-aligned brick, and the     */
/* stiffness of the trilinear brick is a Kronecker sum of 1D operators:      */
/*   K = Lx (x) My (x) Mz  +  Mx (x) Ly (x) Mz  +  Mx (x) My (x) Lz,          */
/* with the 1D linear-element mass M = h [1/3 1/6; 1/6 1/3] and stiffness    */
/* L = (1/h) [1 -1; -1 1].  The elements form a Cartesian product, so the    */
/* assembled matrix is the same Kronecker sum of the assembled 1D matrices.  */
/* At a node with neighbours on both sides along every axis (an interior     */
/* node) those are M(0) = 2h/3, M(+-1) = h/6, L(0) = 2/h, L(+-1) = -1/h, so  */
/* its row holds, at offset (dx, dy, dz) in {-1, 0, 1}^3,                    */
/*   a(dx,dy,dz) = Lx(dx) My(dy) Mz(dz) + Mx(dx) Ly(dy) Mz(dz)                */
/*               + Mx(dx) My(dy) Lz(dz),   h_axis = 1 / n_axis.              */
/* On a cube this is 8h/3 at the centre, 0 at the 6 faces, -h/6 at the 12    */
/* edges and -h/12 at the 8 corners (the assembled stencil the element       */
/* integral gives).  The Dirichlet elimination (orc_dirichlet) turns         */
/* boundary rows into identity rows and drops boundary columns.              */
/* a[(dz+1)*9 + (dy+1)*3 + (dx+1)] = a(dx, dy, dz).                          */
/* ------------------------------------------------------------------------ */
void orc_stencil_coeffs(int nx, int ny, int nz, double a[27])
{
    double h[3] = {1.0 / (double)nx, 1.0 / (double)ny, 1.0 / (double)nz};
    double M[3][3], L[3][3];   /* [axis][offset + 1] */
    for (int ax = 0; ax < 3; ++ax) {
        M[ax][0] = h[ax] / 6.0;
        M[ax][1] = 2.0 * h[ax] / 3.0;
        M[ax][2] = h[ax] / 6.0;
        L[ax][0] = -1.0 / h[ax];
        L[ax][1] = 2.0 / h[ax];
        L[ax][2] = -1.0 / h[ax];
    }
    for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx)
                a[dz * 9 + dy * 3 + dx] = L[0][dx] * M[1][dy] * M[2][dz]
                                        + M[0][dx] * L[1][dy] * M[2][dz]
                                        + M[0][dx] * M[1][dy] * L[2][dz];
}

static int is_boundary_node(int nx, int ny, int nz, int ix, int iy, int iz)
{
    return ix == 0 || ix == nx || iy == 0 || iy == ny || iz == 0 || iz == nz;
}

/* (A x)_i for one row i with the stencil a of orc_stencil_coeffs. */
static double stencil_row(int nx, int ny, int nz, const double a[27], int64_t i, const double *x)
{
    int64_t sx = nx + 1, sxy = (int64_t)(nx + 1) * (ny + 1);
    int ix = (int)(i % sx), iy = (int)((i / sx) % (ny + 1)), iz = (int)(i / sxy);
    if (is_boundary_node(nx, ny, nz, ix, iy, iz))
        return x[i];                                   /* identity row */
    double s = 0.0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (is_boundary_node(nx, ny, nz, ix + dx, iy + dy, iz + dz))
                    continue;                          /* eliminated column */
                s += a[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] *
                     x[node_id(nx, ny, ix + dx, iy + dy, iz + dz)];
            }
    return s;
}

/* (A x)_i of the Dirichlet system for one row i, matrix-free. */
double orc_stencil_row(int nx, int ny, int nz, int64_t i, const double *x)
{
    double a[27];
    orc_stencil_coeffs(nx, ny, nz, a);
    return stencil_row(nx, ny, nz, a, i, x);
}

/* y = A x over all rows, matrix-free. */
void orc_stencil_spmv(int nx, int ny, int nz, const double *x, double *y)
{
    double a[27];
    orc_stencil_coeffs(nx, ny, nz, a);
    int64_t m = orc_num_nodes(nx, ny, nz);
    for (int64_t i = 0; i < m; ++i)
        y[i] = stencil_row(nx, ny, nz, a, i, x);
}

/* Right-hand side of the eliminated system, matrix-free: b_i = g_i on a     */
/* boundary node; elsewhere b_i = 0 - sum over boundary neighbours j of       */
/* a(j - i) g_j (zero source term, the boundary columns moved to the right). */
void orc_stencil_rhs(int nx, int ny, int nz, const double *bc_val, double *b)
{
    double a[27];
    orc_stencil_coeffs(nx, ny, nz, a);
    for (int iz = 0; iz <= nz; ++iz)
        for (int iy = 0; iy <= ny; ++iy)
            for (int ix = 0; ix <= nx; ++ix) {
                int64_t i = node_id(nx, ny, ix, iy, iz);
                if (is_boundary_node(nx, ny, nz, ix, iy, iz)) {
                    b[i] = bc_val[i];
                    continue;
                }
                double s = 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx)
                            if (is_boundary_node(nx, ny, nz, ix + dx, iy + dy, iz + dz))
                                s += a[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] *
                                     bc_val[node_id(nx, ny, ix + dx, iy + dy, iz + dz)];
                b[i] = 0.0 - s;
            }
}
