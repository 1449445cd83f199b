/*
 * fe_cpu_omp.c -- multi-core CPU CG for timing comparisons.
 *
 * MEASUREMENT INFRASTRUCTURE ONLY: bench.py's CPU-baseline leg runs it on the
 * host cores beside the GPU solve.  It is not the oracle (no parity claim
 * rests on it) and the GPU path never calls it.
 *
 * What it computes is the paper's CG module (Sec. 1: DOT, WAXPY, MATVEC;
 * unpreconditioned CG, stop when ||r|| <= tol ||b||) with OpenMP worksharing
 * over rows, in either storage form of Sec. 3.1:
 *   fmt 0  CRS:  y_i = sum_{j = ptr[i]}^{ptr[i+1]-1} val[j] x[col[j]]      (Fig 3.1)
 *   fmt 1  BCRS with 1 x n segments (Fig 3.2/3.3): segment s of row i covers
 *          columns jas[s] .. jas[s] + len - 1 with values val[offsets[s] ..
 *          offsets[s+1] - 1], len = offsets[s+1] - offsets[s]; the inner loop
 *          is specialised on len so one column index serves the whole run.
 * The BCRS arrays are the ones the oracle's csr_to_bcrs builds; val is the CRS
 * value array itself (segments are runs of adjacent CRS entries).
 * Dot products use OpenMP reductions, so their summation order depends on the
 * thread count: results agree with the oracle to rounding, not bitwise.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

static void spmv_crs(int64_t m, const int32_t *ptr, const int32_t *col, const double *val,
                     const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int32_t j = ptr[i]; j < ptr[i + 1]; ++j)
            s += val[j] * x[col[j]];
        y[i] = s;
    }
}

static void spmv_bcrs(int64_t m, const int32_t *ptr, const int32_t *jas, const int32_t *offsets,
                      const double *val, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int32_t g = ptr[i]; g < ptr[i + 1]; ++g) {
            const double *v = val + offsets[g];
            const double *xs = x + jas[g];
            switch (offsets[g + 1] - offsets[g]) {
            case 3: s += v[0] * xs[0] + v[1] * xs[1] + v[2] * xs[2]; break;
            case 2: s += v[0] * xs[0] + v[1] * xs[1]; break;
            case 1: s += v[0] * xs[0]; break;
            default:
                for (int32_t k = 0; k < offsets[g + 1] - offsets[g]; ++k)
                    s += v[k] * xs[k];
            }
        }
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t i = 0; i < n; ++i)
        s += a[i] * b[i];
    return s;
}

static void spmv(int fmt, int64_t m, const int32_t *ptr, const int32_t *idx, const int32_t *offsets,
                 const double *val, const double *x, double *y)
{
    if (fmt == 1)
        spmv_bcrs(m, ptr, idx, offsets, val, x, y);
    else
        spmv_crs(m, ptr, idx, val, x, y);
}

/*
 * CG from the given x (in place).  Returns 0 converged, 1 maxit, 2 breakdown
 * (p.Ap <= 0), -1 out of memory.  *seconds = wall time of the solve (initial
 * residual included, allocation excluded); *threads = OpenMP threads used.
 */
int omp_cg(int64_t m, int fmt, const int32_t *ptr, const int32_t *idx, const int32_t *offsets,
           const double *val, const double *b, double *x, double tol, int maxit, int *iters_out,
           double *relres_out, double *seconds, int *threads)
{
    double *r = (double *)malloc((size_t)m * sizeof(double));
    double *p = (double *)malloc((size_t)m * sizeof(double));
    double *w = (double *)malloc((size_t)m * sizeof(double));
    if (!r || !p || !w) {
        free(r); free(p); free(w);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {   /* first touch by the threads that use them */
        r[i] = 0.0; p[i] = 0.0; w[i] = 0.0;
    }
    *threads = omp_get_max_threads();
    const double t0 = omp_get_wtime();
    int status = 1, k = 0;
    const double bb = dot(m, b, b);
    double rr = 0.0;
    if (bb == 0.0) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i) x[i] = 0.0;
        status = 0;
        goto done;
    }
    spmv(fmt, m, ptr, idx, offsets, val, x, w);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        r[i] = b[i] - w[i];
        p[i] = r[i];
    }
    rr = dot(m, r, r);
    for (;;) {
        if (rr <= tol * tol * bb) { status = 0; break; }
        if (k >= maxit) { status = 1; break; }
        spmv(fmt, m, ptr, idx, offsets, val, p, w);
        const double pw = dot(m, p, w);
        if (!(pw > 0.0)) { status = 2; break; }
        const double alpha = rr / pw;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * w[i];
        }
        const double rr_new = dot(m, r, r);
        const double beta = rr_new / rr;
        rr = rr_new;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            p[i] = r[i] + beta * p[i];
        ++k;
    }
done:
    *seconds = omp_get_wtime() - t0;
    *iters_out = k;
    *relres_out = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    free(r); free(p); free(w);
    return status;
}
