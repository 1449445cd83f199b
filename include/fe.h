/*
 * fe.h -- C ABI of libfe, a GB300 (sm_103a) implementation of the MiniFE
 * steady heat-conduction path studied in "The Research and Optimization of
 * Parallel Finite Element Algorithm based on MiniFE" (arXiv 1505.08023).
 *
 * The problem (paper Sec. 1): the unit cube 0 <= x,y,z <= 1 split into
 * nx x ny x nz trilinear hexahedra, T = 1 on the plane x = 1 and T = 0 on the
 * other faces; the FE system A T = b is solved by unpreconditioned CG.
 *
 * Conventions shared by every call
 *   - Nodes: n_x = nx+1 per x-line, node id i = ix + n_x*(iy + n_y*iz).
 *     Rows of A are nodes; m = n_x n_y n_z.
 *   - Elements: id e = ex + nx*(ey + ny*ez); local node order
 *     (0,0,0),(1,0,0),(1,1,0),(0,1,0),(0,0,1),(1,0,1),(1,1,1),(0,1,1).
 *   - Every pointer argument named d_* is DEVICE memory owned by the caller
 *     (the library allocates nothing, frees nothing and keeps no pointer
 *     after a call returns); h_* are host pointers.  Arrays are dense, C
 *     order, with the lengths stated at each call.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and runs asynchronously unless the call says it synchronises.
 *   - Every call returns an fe_status.  Nothing prints, aborts or traps.
 *     Arguments are checked before anything is enqueued; a CUDA launch or
 *     copy failure returns FE_ERR_CUDA (fe_last_cuda_error() gives the code).
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fe_stream_t; /* same type as cudaStream_t */

typedef enum fe_status {
    FE_OK = 0,
    FE_ERR_ARG = -1,        /* bad size, NULL pointer, unknown enum, misaligned buffer */
    FE_ERR_OVERFLOW = -2,   /* nnz or an index does not fit int32 (N >= 430 on a cube) */
    FE_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    FE_ERR_BREAKDOWN = -4,  /* CG: p.Ap <= 0 or not finite (matrix not SPD, NaN input) */
    FE_ERR_MAXIT = -5,      /* CG: tolerance not met in maxit steps; x holds the iterate */
    FE_ERR_TIMEOUT = -6,    /* CG: a grid barrier waited past its time limit */
    FE_ERR_WORKSPACE = -7   /* workspace smaller than the size query returned */
} fe_status;

/* Storage formats of the assembled matrix. */
typedef enum fe_format {
    FE_FMT_CSR = 0,   /* compressed rows (paper Sec. 3.1, "CRS"): row_ptr, cols, vals */
    FE_FMT_SELL = 1,  /* sliced ELL, 32-row slices, column-major inside a slice */
    FE_FMT_BCRS3 = 2, /* 1x3 blocked rows (the paper's BCRS, Sec. 3.1, with every
                         segment padded to length 3), 32-row slices */
    FE_FMT_VBCRS = 3  /* the paper's BCRS as printed (Sec. 3.1, Fig 3.2/3.3): maximal
                         runs of adjacent columns of variable length, no padding */
} fe_format;

/* Storage type of matrix values. */
typedef enum fe_value_type { FE_VAL_F64 = 0, FE_VAL_F32 = 1, FE_VAL_BF16 = 2 } fe_value_type;

#define FE_SLICE_ROWS 32

/*
 * A matrix on the device, described by plain pointers (all caller-owned).
 *   FE_FMT_CSR   row_ptr[n_rows+1] (int32, row_ptr[n_rows] = nnz), cols[nnz],
 *                vals[nnz]; slice_ptr unused.  n_stored = nnz.
 *   FE_FMT_SELL  slice s holds rows 32s..32s+31 in slots slice_ptr[s] ..
 *                slice_ptr[s+1]-1 (int64, multiples of 32); slot
 *                slice_ptr[s] + 32k + r is entry k of row 32s+r.  cols[] and
 *                vals[] are indexed by slot; padding slots have val 0 and a
 *                valid column.  n_stored = slice_ptr[n_slices].
 *   FE_FMT_BCRS3 like SELL but a slot is a 1x3 segment: cols[slot] is the
 *                first column c of the segment (0 <= c <= n_cols-3) and the
 *                three values multiply x[c], x[c+1], x[c+2].  Values of slot
 *                group g = slice_ptr[s]/32 + k sit at vals[96g + 32t + r],
 *                t = 0, 1, 2 (component), r = row in slice.
 *   FE_FMT_VBCRS the paper's BCRS: a segment is a maximal run of adjacent
 *                columns of a row.  row_ptr[n_rows+1] (int32) holds each
 *                row's first segment ("ptr"), cols[n_stored] each segment's
 *                first column ("jas"), seg_offsets[n_stored+1] (int32) each
 *                segment's first value ("offsets", seg_offsets[n_stored] =
 *                nnz); vals[nnz] is the CSR value array unchanged (values of
 *                segment j at vals[seg_offsets[j] + t], t < its length,
 *                multiplying x[cols[j] + t]).  n_stored = segments (nns).
 * vals has the element type value_type.  n_slices = ceil(n_rows / 32).
 * seg_offsets is used by FE_FMT_VBCRS only (NULL otherwise).
 */
typedef struct fe_matrix {
    int32_t format;           /* fe_format */
    int32_t value_type;       /* fe_value_type */
    int64_t n_rows;
    int64_t n_cols;
    int64_t n_slices;
    int64_t n_stored;         /* nnz (CSR) or slots (SELL, BCRS3) */
    const int32_t *d_row_ptr; /* CSR only */
    const int64_t *d_slice_ptr; /* SELL, BCRS3 */
    const int32_t *d_cols;
    const void *d_vals;
    const int32_t *d_seg_offsets; /* VBCRS only */
} fe_matrix;

/* Sizes of the problem nx x ny x nz (all >= 1). */
typedef struct fe_sizes {
    int64_t n_rows;     /* m = (nx+1)(ny+1)(nz+1) */
    int64_t n_elems;    /* nx ny nz */
    int64_t nnz;        /* (3nx+1)(3ny+1)(3nz+1): full 27-point pattern */
    int64_t n_faces;    /* length of a face-value array (x0,x1,y0,y1,z0,z1) */
    int64_t n_slices;   /* ceil(m / 32) */
} fe_sizes;

/* Sizes for a mesh; FE_ERR_ARG if a dimension is < 1, FE_ERR_OVERFLOW if
 * nnz > INT32_MAX (the int32 row pointer of the CSR form cannot hold it). */
fe_status fe_problem_sizes(int nx, int ny, int nz, fe_sizes *h_out);

/*
 * Mesh processing (paper Sec. 1, mesh module): node coordinates
 * (ix/nx, iy/ny, iz/nz), boundary flag (1 on any face) and prescribed
 * boundary value per node.
 *   d_face_vals  NULL: the paper's data -- 1 on the closed plane x = 1
 *                (edges and corners included), 0 elsewhere.  Otherwise
 *                n_faces values, faces x0, x1, y0, y1, z0, z1 in that order;
 *                an x face is indexed iy + (ny+1) iz, a y face ix + (nx+1) iz,
 *                a z face ix + (nx+1) iy; a later face overwrites an earlier
 *                one on a shared edge.
 *   d_coords     [m][3] double, or NULL (not written: the matrix-free path
 *                needs no coordinates);  d_bc_flag [m] uint8;  d_bc_val [m] double.
 *   d_conn       optional [n_elems][8] int32 element node ids, or NULL.
 * The mesh has no nnz limit (the matrix-free path takes meshes past the CSR
 * form's int32 limit); FE_ERR_OVERFLOW only if d_conn is requested and m
 * exceeds INT32_MAX.
 */
fe_status fe_generate_mesh(int nx, int ny, int nz, const double *d_face_vals,
                           double *d_coords, uint8_t *d_bc_flag, double *d_bc_val,
                           int32_t *d_conn, fe_stream_t stream);

/* Workspace of fe_assemble_csr: 36 doubles per element (upper triangles of
 * the element matrices). */
fe_status fe_assemble_workspace(int nx, int ny, int nz, size_t *h_bytes);

/*
 * Matrix generation and FE assembly (paper Sec. 1; Fig 3.6, Fig 3.7) plus the
 * Dirichlet rows:
 *   - pattern: row i lists its 3x3x3 neighbours that exist (per-axis bounds),
 *     ascending; d_row_ptr[m+1], d_cols[nnz];
 *   - element matrices by 2x2x2 Gauss quadrature from the node coordinates,
 *     summed per row over the incident elements in element-id order
 *     (deterministic; no atomics); zero source, so the load vector is zero;
 *   - Dirichlet rows by symmetric elimination: a boundary row becomes the
 *     identity row with b_i = g_i; elsewhere b_i -= a_ij g_j and a_ij = 0 for
 *     every boundary column j.  The pattern keeps all (3nx+1)(3ny+1)(3nz+1)
 *     entries, zeros included.
 *   d_vals[nnz], d_b[m] double.  d_work: fe_assemble_workspace() bytes,
 *   8-byte aligned; its contents are scratch.
 */
fe_status fe_assemble_csr(int nx, int ny, int nz, const double *d_coords,
                          const uint8_t *d_bc_flag, const double *d_bc_val,
                          int32_t *d_row_ptr, int32_t *d_cols, double *d_vals, double *d_b,
                          void *d_work, size_t work_bytes, fe_stream_t stream);

/*
 * Format conversion at the start of CG (paper Sec. 3.1: CRS is kept for
 * generation and assembly and converted just before the solve).
 *
 * fe_sliced_plan: slot offsets of the 32-row slices for a SELL or BCRS3 copy
 * of the CSR matrix; writes d_slice_ptr[n_slices+1] and *h_n_stored (the
 * call synchronises `stream` to return it).  BCRS3 segments are formed
 * greedily along each row: a segment starts at the first column not yet
 * covered and covers that column and the next two.
 */
fe_status fe_sliced_plan(int32_t format, int64_t n_rows, int64_t n_cols,
                         const int32_t *d_row_ptr, const int32_t *d_cols,
                         int64_t *d_slice_ptr, int64_t *h_n_stored, fe_stream_t stream);

/* Fill a SELL or BCRS3 matrix (format, value_type, sizes and d_slice_ptr set
 * in *dst; d_cols / d_vals point to caller buffers of n_stored entries, with
 * 3 n_stored values for BCRS3) from an FP64 CSR matrix.  Values are rounded
 * to value_type (round to nearest even). */
fe_status fe_convert(const fe_matrix *src_csr, const fe_matrix *dst, fe_stream_t stream);

/*
 * The paper's BCRS (Sec. 3.1) from a CSR matrix with sorted columns: a new
 * segment starts at the first entry of a row and wherever a column is not the
 * previous column + 1.  fe_vbcrs_plan writes the segment row pointer
 * d_seg_ptr[n_rows+1] and the segment count to *h_nns (synchronises
 * `stream`; d_work: fe_vbcrs_workspace() bytes of scratch, 8-byte aligned);
 * fe_vbcrs_fill then writes d_jas[nns] and d_seg_offsets[nns+1].  The value
 * array is the CSR one (or a rounded copy of it, fe_round_values): the VBCRS
 * descriptor points at it.  Errors: FE_ERR_ARG (not CSR, null or misaligned
 * pointers), FE_ERR_WORKSPACE, FE_ERR_OVERFLOW (nns above int32).
 */
fe_status fe_vbcrs_workspace(int64_t n_rows, size_t *h_bytes);
fe_status fe_vbcrs_plan(const fe_matrix *csr, int32_t *d_seg_ptr, void *d_work, size_t work_bytes,
                        int64_t *h_nns, fe_stream_t stream);
fe_status fe_vbcrs_fill(const fe_matrix *csr, const int32_t *d_seg_ptr, int32_t *d_jas,
                        int32_t *d_seg_offsets, fe_stream_t stream);

/* Round an FP64 array to value_type (FE_VAL_F32 or FE_VAL_BF16), nearest even:
 * a CSR copy of the matrix with lower-precision values. */
fe_status fe_round_values(int64_t n, const double *d_src, int32_t value_type, void *d_dst,
                          fe_stream_t stream);

/* SpMV y = A x (paper Fig 3.1 / Fig 3.2) in any format and value type,
 * FP64 vectors and FP64 accumulation.  d_x[n_cols], d_y[n_rows]. */
fe_status fe_spmv(const fe_matrix *A, const double *d_x, double *d_y, fe_stream_t stream);

/* The same with FP32 vectors and FP32 accumulation (inner solve of the
 * mixed-precision form). */
fe_status fe_spmv_f32(const fe_matrix *A, const float *d_x, float *d_y, fe_stream_t stream);

/* Result of a CG solve. */
typedef struct fe_cg_result {
    int32_t status;      /* fe_status of the solve */
    int32_t iterations;  /* CG steps taken */
    double relres;       /* ||r_k|| / ||b|| of the recursive residual */
    double bnorm;        /* ||b|| */
} fe_cg_result;

/* Workspace of fe_cg_solve and fe_cg_solve_form for matrix A: four vectors
 * (r, w and two p buffers) of 32 * n_slices doubles plus the reduction and
 * barrier block (about 128 KiB). */
fe_status fe_cg_workspace(const fe_matrix *A, size_t *h_bytes);

/*
 * Unpreconditioned CG on A x = b (paper Sec. 1: MATVEC, DOT, WAXPY), textbook
 * form, the whole loop in one persistent cooperative kernel: each step makes
 * one pass over the matrix (w = A p with p.w fused into the SpMV epilogue),
 * then x += alpha p, r -= alpha w with r.r fused, then p = r + beta p; dot
 * products are reduced in a fixed order, so a rerun gives identical bits.
 *   Stop when ||r_k|| <= tol ||b|| (checked before the first step and after
 *   each update) or after maxit steps; b = 0 returns x = 0.
 *   d_x[m]: start vector in, iterate out (d_b, d_x 16-byte aligned).  d_work: fe_cg_workspace() bytes,
 *   256-byte aligned, scratch.  timeout_s: limit on any one grid-barrier
 *   wait (<= 0: 2 s); past it every block exits and the status is
 *   FE_ERR_TIMEOUT.
 *   Synchronises `stream` and fills *h_result (required); returns its status.
 */
fe_status fe_cg_solve(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                      double timeout_s, void *d_work, size_t work_bytes,
                      fe_cg_result *h_result, fe_stream_t stream);

/*
 * fe_cg_solve with the kernel form chosen by the caller (paper Sec. 1, the
 * same CG iteration; the forms differ only in how a step is cut into grid
 * phases).  fe_cg_solve is this call with FE_CG_AUTO.
 *   FE_CG_THREE_PHASE: SpMV with p.w; r update with r.r; x and p update --
 *     three grid barriers per step, no work repeated.
 *   FE_CG_TWO_PHASE: the x and p update of a step is folded into the next
 *     step's SpMV (p = r + beta p_old formed at every gathered column, p
 *     double-buffered) -- two barriers per step, one more FMA and two vector
 *     loads per stored entry; for meshes whose step time is set by barrier
 *     latency.
 *   FE_CG_RESIDENT: the two-phase step with the matrix held in registers:
 *     for FP64 BCRS3 or sliced-ELL matrices of at most SMs * 8 slices (one
 *     slice per warp, one block of 8 warps per SM; 38,912 rows on 152 SMs),
 *     each warp loads its slice's entries once and keeps its rows' x, r, p
 *     and w in registers for the whole solve (x is stored once, at the end);
 *     for matrices that do not qualify: FE_ERR_ARG.
 *   FE_CG_AUTO: the resident form when A qualifies, else the two-phase form
 *     while the grid holds at most one 32-row slice per warp
 *     (n_slices <= SMs * 4 * 8), else the three-phase form.
 *   The three- and two-phase forms perform the same floating-point operations
 *   in the same order and return identical bits; the resident form sums the
 *   dot products' per-thread partials per row instead of per 16-byte pack,
 *   so its bits can differ in the last place.  Other form values:
 *   FE_ERR_ARG.  Arguments, workspace, result and errors otherwise as
 *   fe_cg_solve.
 */
#define FE_CG_AUTO 0
#define FE_CG_THREE_PHASE 1
#define FE_CG_TWO_PHASE 2
#define FE_CG_RESIDENT 3
fe_status fe_cg_solve_form(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                           double timeout_s, int form, void *d_work, size_t work_bytes,
                           fe_cg_result *h_result, fe_stream_t stream);

/* Workspace of fe_cg_solve_sr: four vectors (r, p, w, s) of 32 * n_slices
 * doubles plus the reduction and barrier block. */
fe_status fe_cg_sr_workspace(const fe_matrix *A, size_t *h_bytes);

/*
 * Single-reduction CG (Chronopoulos and Gear, 1989, s = 1): the same Krylov
 * iterates as fe_cg_solve in exact arithmetic (the paper's CG module,
 * Sec. 1), reorganised so that each step needs one grid reduction: w = A r
 * with r.r and w.r fused into the SpMV epilogue, then
 *   beta = gamma_k / gamma_{k-1},  p.Ap = delta_k - beta gamma_k / alpha_{k-1},
 *   alpha = gamma_k / p.Ap,  p = r + beta p,  s = w + beta s (s = A p),
 *   x += alpha p,  r -= alpha s.
 * Two grid barriers per step instead of three (faster where barriers
 * dominate: small meshes); one extra vector and one extra FMA per row.
 * Arguments, stopping rule, timeout, determinism and result as fe_cg_solve
 * (d_work: fe_cg_sr_workspace() bytes).  When the curvature recurrence gives
 * p.Ap <= 0 (rounding near convergence) the step restarts the direction
 * (beta = 0, p.Ap = r.Ar); FE_ERR_BREAKDOWN when r.Ar <= 0.
 */
fe_status fe_cg_solve_sr(const fe_matrix *A, const double *d_b, double *d_x, double tol, int maxit,
                         double timeout_s, void *d_work, size_t work_bytes,
                         fe_cg_result *h_result, fe_stream_t stream);

/* Result of a mixed-precision solve. */
typedef struct fe_mixed_result {
    int32_t status;            /* fe_status of the solve */
    int32_t outer_iterations;  /* refinement steps (inner solves) */
    int32_t inner_iterations;  /* FP32 CG steps over all inner solves */
    int32_t reserved;
    double relres;             /* true FP64 ||b - A64 x|| / ||b|| at exit */
    double bnorm;              /* ||b|| */
} fe_mixed_result;

/* Workspace of fe_cg_solve_mixed for the low-precision matrix A_lo: five FP32
 * vectors of 32 * n_slices entries plus reduction blocks (either mode). */
fe_status fe_cg_mixed_workspace(const fe_matrix *A_lo, size_t *h_bytes);

/* Modes of the mixed-precision solve. */
typedef enum fe_mixed_mode {
    FE_MIXED_RELIABLE = 0,  /* one persistent kernel, refinement steps keep the search direction */
    FE_MIXED_RESTART = 1    /* host loop of restarted inner solves */
} fe_mixed_mode;

/*
 * Mixed-precision form of the solve (not in the paper; it must reach the same
 * FP64 true residual as the FP64 path).  A_lo holds the matrix values in FP32 or BF16 (any format); the
 * Krylov iteration runs in FP32 with FP32 accumulation on A_lo; the residual
 * recompute r = b - A64 x (A64: FP64 values, any format), the refinement
 * update x += d and every global dot product are FP64.  The stopping test is
 * the true FP64 residual: ||b - A64 x|| <= tol ||b||.
 *
 *   FE_MIXED_RELIABLE: one persistent cooperative kernel.  The FP32 CG
 *     accumulates a correction d; each time its residual has fallen by the
 *     factor inner_tol since the last refinement step (or meets tol), the
 *     kernel sets x += d (FP64), recomputes r = b - A64 x (FP64) as the FP32
 *     residual and continues with the same search direction.  max_outer caps
 *     the refinement steps, max_inner the FP32 CG steps; four refinement
 *     steps in a row that do not halve the true residual (a step is forced
 *     after 256 FP32 steps without one) also end the solve
 *     (FE_ERR_MAXIT): the low-precision operator is then too far from A64
 *     (value error x condition number ~ 1), e.g. BF16 values on strongly
 *     non-cubic elements.  A_lo must not be FP64.  A BCRS3 A_lo whose d_cols
 *     and d_vals start on 16-byte boundaries is streamed into shared memory
 *     by bulk copies (46 KB of shared memory per block for BF16 values,
 *     74 KB for FP32); other alignments are read by thread loads.  Both give
 *     bitwise the same result.
 *   FE_MIXED_RESTART: repeat { r = b - A64 x; solve A_lo d = r by the FP32
 *     persistent CG from d = 0 to ||r_in|| <= inner_tol ||r|| or max_inner
 *     steps; x += d } at most max_outer times.
 *
 *   d_b, d_x (16-byte aligned): right-hand side; start in, solution out.
 *   d_work: fe_cg_mixed_workspace() bytes, 256-byte aligned.  Synchronises
 *   `stream` (once per solve in RELIABLE mode, once per step in RESTART).
 *   h_result->outer_iterations counts refinement steps, inner_iterations the
 *   FP32 CG steps, relres is the last FP64 true residual.
 */
fe_status fe_cg_solve_mixed(const fe_matrix *A64, const fe_matrix *A_lo, const double *d_b,
                            double *d_x, double tol, int mode, int max_outer, double inner_tol,
                            int max_inner, double timeout_s, void *d_work, size_t work_bytes,
                            fe_mixed_result *h_result, fe_stream_t stream);

/*
 * fe_cg_solve without a workspace argument, for callers that cannot allocate
 * device memory when they solve (a latency-critical loop where cudaMalloc's
 * implicit device synchronisation is unacceptable, or a plugin whose host
 * framework owns all device memory).  The paper has no counterpart: this is
 * a packaging variant of the same solve.
 *   The solver's scratch comes from a fixed array inside the library (about
 *   8.5 MB, held on every GPU that loads the library until the process
 *   exits), so A may have at most FE_NOALLOC_MAX_ROWS rows (32 * n_slices <=
 *   FE_NOALLOC_MAX_ROWS, e.g. meshes up to 63 x 63 x 63 elements); larger A
 *   returns FE_ERR_WORKSPACE before anything is enqueued.
 *   Every call looks up that array's device address on the current device
 *   (a host-side query that allocates nothing), so the address stays valid
 *   after a cudaDeviceReset.
 *   All calls share the one array: calls whose work overlaps on the GPU (two
 *   streams, two host threads) race and give undefined results; serialise
 *   them.  Each call re-initialises the part that must start at zero.
 *   Arguments, results and synchronisation are those of fe_cg_solve.
 */
#define FE_NOALLOC_MAX_ROWS 262144
fe_status fe_cg_solve_noalloc(const fe_matrix *A, const double *d_b, double *d_x, double tol,
                              int maxit, double timeout_s, fe_cg_result *h_result,
                              fe_stream_t stream);

/*
 * Batched form (an extension; the paper solves one system): many
 * independent CG solves -- meshes of different sizes, different boundary data
 * -- in one persistent cooperative launch.  System i is A[i] x_i = b_i; every
 * A[i] is FP64 with one common format (FE_FMT_BCRS3 or FE_FMT_SELL).  Systems
 * whose descriptors point to the same arrays share the matrix and are solved
 * together as an SpMM over up to `krhs` (1, 2 or 4) right-hand sides, so each
 * matrix slot is read once per chunk.  Each system keeps its own alpha, beta,
 * stopping test (||r|| <= tol ||b||) and status, exactly as fe_cg_solve; a
 * converged system leaves the work list and the remaining work is
 * re-partitioned over all blocks.  Dot products are summed in a fixed order.
 *
 * fe_cg_batched_plan   checks the systems, groups them, writes the work tables
 *                      into d_work and fills *h_plan (synchronises `stream`).
 *                      method: FE_BATCH_TEXTBOOK (three grid barriers per
 *                      step) or FE_BATCH_SINGLE_REDUCTION (the recurrences of
 *                      fe_cg_solve_sr, two barriers per step).
 *                      blocks_per_sm: 0 = the most that fit.
 * fe_cg_batched_launch enqueues the solve (a memset and one cooperative
 *                      kernel; no host synchronisation, no allocation), so it
 *                      can be captured in a CUDA graph and replayed.
 * fe_cg_batched_results copies the per-system results into h_results[i]
 *                      (caller's order; synchronises) and returns the first
 *                      non-OK status, or FE_OK.
 * fe_cg_solve_batched  plan (FE_BATCH_TEXTBOOK) + launch + results.
 * d_x[i] (16-byte aligned): start vectors in, solutions out.  At most FE_BATCH_MAX_SYSTEMS
 * systems; FE_ERR_ARG if a block would have to reduce more than 32 systems.
 */
#define FE_BATCH_MAX_SYSTEMS 256
#define FE_BATCH_TEXTBOOK 0
#define FE_BATCH_SINGLE_REDUCTION 1
typedef struct fe_batch_plan {
    int32_t format, krhs, n_systems, n_chunks, grid, max_blocks, method;
    void *d_work;
    size_t work_bytes;
    int32_t slot_of[FE_BATCH_MAX_SYSTEMS];  /* caller's index -> internal slot */
} fe_batch_plan;

fe_status fe_cg_batched_workspace(int n_systems, const fe_matrix *A, size_t *h_bytes);
fe_status fe_cg_batched_plan(int n_systems, const fe_matrix *A, const double *const *d_b,
                             double *const *d_x, int krhs, int method, int blocks_per_sm,
                             void *d_work, size_t work_bytes, fe_batch_plan *h_plan,
                             fe_stream_t stream);
fe_status fe_cg_batched_launch(const fe_batch_plan *plan, double tol, int maxit, double timeout_s,
                               fe_stream_t stream);
fe_status fe_cg_batched_results(const fe_batch_plan *plan, fe_cg_result *h_results,
                                fe_stream_t stream);
fe_status fe_cg_solve_batched(int n_systems, const fe_matrix *A, const double *const *d_b,
                              double *const *d_x, double tol, int maxit, int krhs,
                              double timeout_s, void *d_work, size_t work_bytes,
                              fe_cg_result *h_results, fe_stream_t stream);

/*
 * Learned warm start (an extension, not in the paper).  Kernels of a
 * 3-D convolutional encoder-decoder that maps the boundary data of a mesh to
 * a CG start vector, and of its training.  Volumes are FP32 arrays
 * [C][D][H][W] (W fastest) on one sample; dims arrays are {D, H, W}.
 * Weights of a 3x3x3 layer: FP32 master [cin][27][cout] (tap t = 9 dz + 3 dy
 * + dx); the kernels read a BF16 copy (d_w: bfloat16 bits) and accumulate in
 * FP32.  A layer in "gather" form computes
 *   out[co][u] = bias[co] + sum_ci sum_t W[ci][t][co] in[ci][src(u, t)]
 * with per axis src = u + d - 1 (FE_NN_S1), 2u + d - 1 (FE_NN_S2, D_out =
 * (D_in - 1)/2 + 1) or (u + 1 - d)/2 where integral (FE_NN_T2, D_out =
 * 2 (D_in - 1) + 1); zero outside the input grid; `relu` clamps at zero.
 * The data gradient of S1 is S1 with fe_nn_pack_weights(transpose=1,
 * flip=1); of S2 it is T2 and of T2 it is S2 with (transpose=1, flip=0).
 */
#define FE_NN_S1 0
#define FE_NN_S2 1
#define FE_NN_T2 2

fe_status fe_nn_conv3d(int mode, const float *d_in, int cin, const int *h_dims_in, const void *d_w,
                       const float *d_bias, float *d_out, int cout, const int *h_dims_out,
                       int relu, fe_stream_t stream);
/* BF16 copies of FP32 master weights [cin][27][cout]: transpose=0 keeps the
 * layout; transpose=1 writes [cout][27][cin] (taps reversed if flip=1). */
fe_status fe_nn_pack_weights(const float *d_w, int cin, int cout, int transpose, int flip,
                             void *d_out, fe_stream_t stream);
/* Stride-1 3x3x3 convolution on the tensor cores (tcgen05.mma, FP32
 * accumulators in tensor memory); not in the paper, part of the warm start.
 * Same definition as fe_nn_conv3d(FE_NN_S1, ...), dims_out = dims_in, except
 * that the activations are rounded to BF16 (nearest even) before the
 * products: |out - exact| <= (2^-8 + 2 K 2^-24) sum |w| |x|, K = 27 cin + 1.
 *   d_img: the weights as fe_nn_pack_weights_mma laid them out
 *   (fe_nn_mma_image_bytes bytes, 16-byte aligned); cout must be 16, 32 or 64.
 *   d_bias may be NULL; relu != 0 applies ReLU.  Allocates nothing; enqueues
 *   one kernel on `stream`.  A block whose bounded wait for the tensor cores
 *   runs out (1 s) stops and raises a flag that fe_nn_tc_check reports. */
fe_status fe_nn_mma_image_bytes(int cin, int cout, size_t *h_bytes);
/* Lay out BF16 weights [cin][27][cout] (from fe_nn_pack_weights, either copy)
 * as the tensor-core operand image: per 16-channel chunk kc, per tap t, the
 * 8-channel groups kg as cout rows of 16 bytes (channels past cin are 0). */
fe_status fe_nn_pack_weights_mma(const void *d_w16, int cin, int cout, void *d_img,
                                 fe_stream_t stream);
fe_status fe_nn_conv3d_s1_tc(const float *d_in, int cin, const int *h_dims, const void *d_img,
                             const float *d_bias, float *d_out, int cout, int relu,
                             fe_stream_t stream);
/* Transposed stride-2 convolution (fe_nn_conv3d(FE_NN_T2, ...)) on the tensor
 * cores, same contract and bound as fe_nn_conv3d_s1_tc; h_dims_out must be
 * 2 (h_dims_in - 1) + 1.  The eight output parity classes are separate
 * accumulators; each (class, tap) pair is one MMA on the shifted input box. */
fe_status fe_nn_conv3d_t2_tc(const float *d_in, int cin, const int *h_dims_in, const void *d_img,
                             const float *d_bias, float *d_out, int cout, const int *h_dims_out,
                             int relu, fe_stream_t stream);
/* Stride-2 convolution (fe_nn_conv3d(FE_NN_S2, ...)) on the tensor cores,
 * same contract and bound; h_dims_out must be (h_dims_in - 1) / 2 + 1.  The
 * fine input box is staged as eight parity sub-boxes on the coarse lattice. */
fe_status fe_nn_conv3d_s2_tc(const float *d_in, int cin, const int *h_dims_in, const void *d_img,
                             const float *d_bias, float *d_out, int cout, const int *h_dims_out,
                             int relu, fe_stream_t stream);
/* Tensor-core convolution (mode FE_NN_S1, FE_NN_S2 or FE_NN_T2) reading its
 * input as BF16 in the 8-channel-interleaved layout [ceil(cin/8)][D][H][W][8]
 * that fe_nn_to_bf16i writes (fe_nn_bf16i_bytes bytes, 16-byte aligned).  The
 * input box of each 16-channel chunk is staged by tensor-map (TMA) loads with
 * zero fill outside the grid; otherwise as fe_nn_conv3d_{s1,s2,t2}_tc (same
 * result bits: the FP32 kernels round the same values to BF16).  A TMA box
 * spans at most 256 points per axis: input width <= 254 (stride 1), <= 255
 * (transposed), output width <= 127 (stride 2); wider grids get FE_ERR_ARG. */
fe_status fe_nn_bf16i_bytes(int c, const int *h_dims, size_t *h_bytes);
fe_status fe_nn_to_bf16i(const float *d_in, int c, const int *h_dims, void *d_out, fe_stream_t stream);
fe_status fe_nn_conv3d_tc_bf16i(int mode, const void *d_in16, int cin, const int *h_dims_in, const void *d_img,
                                const float *d_bias, float *d_out, int cout, const int *h_dims_out, int relu,
                                fe_stream_t stream);
/* Synchronises the device; *h_flag = 1 if a tensor-core kernel gave up a wait
 * since the last call (then clears the flag), else 0. */
fe_status fe_nn_tc_check(int *h_flag);

/* Scratch of fe_nn_conv3d_weight_grad: per-split partial sums; h_splits gets
 * the split count.  stride 1 or 2; (ca, dims_a) describe the correlation's
 * first operand (dY for S1/S2, X for T2). */
fe_status fe_nn_corr_workspace(int stride, int ca, const int *h_dims_a, int cb, size_t *h_bytes,
                               int *h_splits);
/* dW[ci][t][co] = d loss / d W of a layer given its input X and the gradient
 * dY of its output (FP32), summed over voxel tiles in a fixed order. */
fe_status fe_nn_conv3d_weight_grad(int mode, const float *d_x, int cin, const int *h_dims_in,
                                   const float *d_dy, int cout, const int *h_dims_out, float *d_dw,
                                   float *d_work, size_t work_bytes, fe_stream_t stream);
/* The same weight gradient on the tensor cores (tcgen05): per tap a GEMM over
 * the voxels, operands rounded to BF16 (nearest even), FP32 accumulation in
 * tensor memory, per-block partials summed in a fixed order.  d_work
 * (fe_nn_wgrad_tc_workspace() bytes, 16-byte aligned) holds the partials and,
 * unless the grid is too wide for a 256-point box, a BF16 8-channel-interleaved
 * copy of the second operand (X for S1/S2, dY for T2) that the kernel stages
 * with tensor-map box loads.  The channels of the layer's input (S1,
 * S2) or output (T2) must be 16, 32 or 64, the others at most 128; other
 * shapes: FE_ERR_ARG (the CUDA-core fe_nn_conv3d_weight_grad takes them). */
fe_status fe_nn_wgrad_tc_workspace(int mode, int cin, const int *h_dims_in, int cout, const int *h_dims_out,
                                   size_t *h_bytes);
fe_status fe_nn_conv3d_weight_grad_tc(int mode, const float *d_x, int cin, const int *h_dims_in,
                                      const float *d_dy, int cout, const int *h_dims_out, float *d_dw,
                                      float *d_work, size_t work_bytes, fe_stream_t stream);
/* db[c] = sum over the volume of dY[c] (bias gradient), fixed order. */
fe_status fe_nn_channel_sum(const float *d_dy, int c, const int *h_dims, float *d_db,
                            fe_stream_t stream);
/* dy[i] = 0 where y[i] <= 0 (backward of a fused ReLU). */
fe_status fe_nn_relu_bwd(const float *d_y, float *d_dy, size_t n, fe_stream_t stream);
/* y += a x. */
fe_status fe_nn_axpy(float a, const float *d_x, float *d_y, size_t n, fe_stream_t stream);
/* 1x1x1 head out[u] = b + sum_c w[c] h[c][u] (w: c bfloat16), and its
 * backward (d_work: (c+1) * 64 floats). */
fe_status fe_nn_head(const float *d_h, int c, const int *h_dims, const void *d_w, const float *d_b,
                     float *d_out, fe_stream_t stream);
fe_status fe_nn_head_bwd(const float *d_h, int c, const int *h_dims, const void *d_w,
                         const float *d_dout, float *d_dh, float *d_dw, float *d_db, float *d_work,
                         size_t work_bytes, fe_stream_t stream);
/* Mean squared error over interior nodes (bc_flag == 0): d_dpred = 2 scale
 * (pred - target) inside, 0 on boundary nodes; d_loss_parts[n_parts] get
 * partial sums of the squared error (n_parts blocks, fixed order). */
fe_status fe_nn_mse(const float *d_pred, const float *d_target, const uint8_t *d_bc_flag, size_t n,
                    float scale, float *d_dpred, float *d_loss_parts, int n_parts,
                    fe_stream_t stream);
/* One Adam step on FP32 master weights; lr_t includes the bias corrections. */
fe_status fe_nn_adam(float *d_w, const float *d_g, float *d_m, float *d_v, size_t n, float lr_t,
                     float beta1, float beta2, float eps, fe_stream_t stream);
/* Network input from the mesh: d_x[2][m] = (boundary value or 0, boundary flag). */
fe_status fe_warmstart_input(const uint8_t *d_bc_flag, const double *d_bc_val, size_t n, float *d_x,
                             fe_stream_t stream);
/* CG start vector: prescribed value on boundary nodes, the prediction inside. */
fe_status fe_warmstart_output(const float *d_pred, const uint8_t *d_bc_flag, const double *d_bc_val,
                              size_t n, double *d_x0, fe_stream_t stream);

/*
 * Warm-start inference in one call (an extension, not in the paper): the
 * boundary data of an n_nodes^3 mesh (bc_flag, bc_val, as fe_generate_mesh
 * writes them) in, the CG start vector d_x0 (n_nodes^3 doubles) out, through
 * the 4-level encoder-decoder with channels h_channels[0..3]:
 *   e0 = relu(S1(x)), d1 = relu(S2(e0)), e1 = relu(S1(d1)), ..., e3 = relu(S1(d3)),
 *   s2 = relu(T2(e3) + e2), f2 = relu(S1(s2)), s1, f1, s0, f0 likewise,
 *   pred = b_h + sum_c w_h[c] f0[c]; x0 = bc_val on boundary nodes, pred inside.
 * n_nodes - 1 must be a multiple of 8 (levels n_l = (n_nodes - 1)/2^l + 1).
 * d_blob (256-byte aligned) holds, in the layer order e0 d1 e1 d2 e2 d3 e3 u2
 * f2 u1 f1 u0 f0, each layer's bias FP32 [cout] and weights BF16
 * [cin][27][cout] (the fe_nn_pack_weights forward layout), then the head
 * weights BF16 [c0] and bias FP32 [1]; fe_warmstart_blob_layout gives the 28
 * section offsets (each 256-byte aligned) and the size.  tensor_cores != 0
 * runs every layer with >= 16 input and 16/32/64 output channels on the
 * tensor cores (BF16 activations: each such layer's input is converted by
 * fe_nn_to_bf16i into a scratch area of the workspace and staged by TMA), the
 * others on CUDA cores.  d_work: fe_warmstart_workspace bytes, 256-byte aligned.  Enqueues on `stream`,
 * allocates nothing.
 */
fe_status fe_warmstart_blob_layout(const int *h_channels, size_t *h_offsets /* 28 or NULL */,
                                   size_t *h_bytes);
fe_status fe_warmstart_workspace(int n_nodes, const int *h_channels, size_t *h_bytes);
fe_status fe_warmstart_infer(int n_nodes, const int *h_channels, const void *d_blob,
                             const uint8_t *d_bc_flag, const double *d_bc_val, double *d_x0,
                             void *d_work, size_t work_bytes, int tensor_cores, fe_stream_t stream);

/* Fault injection for tests of the barrier time limit: the next fe_cg_solve
 * or fe_cg_solve_sr on the calling thread has block 0 skip its arrival at grid barrier number
 * barrier_index (0 = the barrier after the initial residual), so every
 * block's bounded wait runs out and the solve returns FE_ERR_TIMEOUT with
 * the GPU context intact.  -1 clears it.  Nothing faults, traps or hangs. */
fe_status fe_inject_barrier_stall(int barrier_index);

/* True relative residual ||b - A x|| / ||b|| (||b - A x|| if b = 0), FP64,
 * with A's stored values.  d_work: at least FE_RESID_WORK_BYTES, 8-byte
 * aligned (per-block partial sums).  Synchronises `stream`. */
#define FE_RESID_WORK_BYTES (65536 + 64)
fe_status fe_true_relres(const fe_matrix *A, const double *d_b, const double *d_x,
                         void *d_work, size_t work_bytes, double *h_relres, fe_stream_t stream);

/*
 * Matrix-free operator (an extension beside the paper's stored CRS/BCRS
 * formats, Sec. 3.1): the same Dirichlet system as fe_assemble_csr on the
 * nx x ny x nz box mesh, applied without a stored matrix.  The trilinear
 * brick's stiffness is the Kronecker sum Lx(x)My(x)Mz + Mx(x)Ly(x)Mz +
 * Mx(x)My(x)Lz of 1D linear-element mass and stiffness, and so is the
 * assembled matrix; a row whose node is not on a face holds, at offset
 * (dx, dy, dz) in {-1,0,1}^3,
 *   a = Lx(dx) My(dy) Mz(dz) + Mx(dx) Ly(dy) Mz(dz) + Mx(dx) My(dy) Lz(dz),
 *   M(0) = 2h/3, M(+-1) = h/6, L(0) = 2/h, L(+-1) = -1/h, h = 1/n per axis
 * (on a cube: 8h/3 centre, 0 faces, -h/6 edges, -h/12 corners).  Rows of
 * boundary nodes are identity rows; boundary columns are eliminated.  The
 * values equal the element-integral ones up to rounding (the stored matrix
 * also holds ~1e-18 quadrature residues where the exact value is 0).
 * Node ids as fe_generate_mesh; m = (nx+1)(ny+1)(nz+1) may exceed the int32
 * limit of the CSR form (indices are 64-bit).  Vectors are m doubles,
 * 8-byte aligned; FE_ERR_ARG on bad sizes, null or aliased pointers.
 *
 * fe_stencil_spmv: d_y = A d_x (d_y must not alias d_x).
 * fe_stencil_rhs:  d_b = the right-hand side of the eliminated system: the
 *   prescribed value on boundary nodes, 0 - sum_j a_ij g_j over boundary
 *   neighbours j elsewhere (zero source term).  d_bc_val: fe_generate_mesh's.
 * fe_stencil_cg_solve: textbook CG on A x = b, stopping rule, status codes,
 *   result and bounded barriers as fe_cg_solve; d_x holds the start vector.
 *   d_work: fe_stencil_cg_workspace bytes (four m-vectors plus the reduction
 *   block), 256-byte aligned.  Synchronises `stream`.
 * fe_stencil_true_relres: ||b - A x|| / ||b|| (||b - A x|| if b = 0) with the
 *   matrix-free A; d_work as fe_stencil_cg_solve (its contents are scratch).
 */
fe_status fe_stencil_spmv(int nx, int ny, int nz, const double *d_x, double *d_y, fe_stream_t stream);
fe_status fe_stencil_rhs(int nx, int ny, int nz, const double *d_bc_val, double *d_b, fe_stream_t stream);
fe_status fe_stencil_cg_workspace(int nx, int ny, int nz, size_t *h_bytes);
fe_status fe_stencil_cg_solve(int nx, int ny, int nz, const double *d_b, double *d_x, double tol,
                              int maxit, double timeout_s, void *d_work, size_t work_bytes,
                              fe_cg_result *h_result, fe_stream_t stream);
fe_status fe_stencil_true_relres(int nx, int ny, int nz, const double *d_b, const double *d_x,
                                 void *d_work, size_t work_bytes, double *h_relres,
                                 fe_stream_t stream);

/* CUDA error code of the last FE_ERR_CUDA on this thread (0 if none). */
int fe_last_cuda_error(void);

/* Version string of the library. */
const char *fe_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
