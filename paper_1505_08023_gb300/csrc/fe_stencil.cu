// fe_stencil.cu -- the Dirichlet system's operator applied without a stored
// matrix (matrix-free), and the CG solve built on it.  An extension beside the
// paper's stored CRS/BCRS formats (Sec. 3.1): same operator, same CG (Sec. 1),
// no matrix stream.
//
// On the box mesh every element is the same axis-aligned brick, and the
// trilinear brick's stiffness is the Kronecker sum
//   Lx (x) My (x) Mz + Mx (x) Ly (x) Mz + Mx (x) My (x) Lz
// of 1D linear-element mass and stiffness matrices.  The elements form a
// Cartesian product, so the assembled matrix is the same Kronecker sum of the
// assembled 1D matrices, and a row whose node has neighbours on both sides
// along every axis holds, at offset (dx, dy, dz),
//   a = Lx(dx) My(dy) Mz(dz) + Mx(dx) Ly(dy) Mz(dz) + Mx(dx) My(dy) Lz(dz),
// M(0) = 2h/3, M(+-1) = h/6, L(0) = 2/h, L(+-1) = -1/h, h = 1/n per axis.
// a depends on |dx|, |dy|, |dz| only: eight classes c[k], k = |dx| + 2|dy| +
// 4|dz|.  Boundary rows are identity rows and boundary columns are
// eliminated (their values read as 0), as in the assembled system.
//
// Interior rows: a block of 8 warps owns a 32 x 16 (x, y) column of interior
// nodes (two rows per warp) and marches along z through a range of planes.
// Each plane is staged in shared memory with a one-node halo (boundary and
// out-of-range nodes as 0; double-buffered, the next plane's loads in flight
// while this one is used), and every thread forms the plane sums of its two
// nodes:  X (centre), Sx = x(-1) + x(+1), Sy = y(-1) + y(+1), D = the four
// in-plane diagonal neighbours, taken as Sx of the rows above and below (the
// staged rows' Sx go through shared memory: one add per row instead of
// three; a thread's two rows take each other's X and Sx from registers).
// The row of plane z is
//   y = c0 X + c1 Sx + c2 Sy + c3 D              (plane z)
//     + Q(z-1) + Q(z+1),  Q = c4 X + c5 Sx + c6 Sy + c7 D   (planes z-1, z+1)
// with Q carried in registers from plane to plane.  On a cube the face
// classes vanish (c1 = c2 = c4 = 0) and the three edge classes agree, so
//   y = c0 X + c3 D + P(z-1) + P(z+1),  P = c3 (Sx + Sy) + c7 D:
// 9.125 FP64 operations per row (Sx 1.125 with the halo rows, Sy 1, D 1,
// P 3, the row 3) where the stored matrix takes 27 FMAs.  The
// work (interior columns x interior planes) is cut into equal contiguous
// ranges, one per block, so every block marches the same number of planes.
// Boundary rows (y = x) are a separate row loop.
//
// CG (textbook Hestenes-Stiefel, as fe_cg_solve) in two phases per step:
//   A  p = r + beta p_old and x += alpha_old p_old, fused into the staging of
//      the SpMV operand (p is double-buffered: neighbours' halos still read
//      p_old), w = A p, p.w in the epilogue
//   B  r -= alpha w, r.r
// so a step streams 72 bytes of vectors per row and takes two grid
// reductions, with the same bounded barrier and fixed-order sums as k_cg.
#include "fe_cg_common.cuh"
#include "fe_stencil_geom.cuh"

namespace fe {

static_assert(kStWarps == kCgWarps && kStThreads == kCgThreads, "tiles are cut for the CG block");

// Pointers of one operator pass.
struct StencilIO {
    const double *in;     // operand (plain pass) or r (CG pass)
    const double *pold;   // CG pass: p of the previous step; nullptr on the first step
    double *pnew;         // CG pass: p of this step, written for every row
    double *x;            // CG pass: x += alpha_old p_old (with pold)
    double *out;          // A times the operand
    double beta, alpha_old;
};

// One column of interior rows, planes zlo .. zhi-1 (1-based interior
// planes); returns the thread's partial of operand . (A operand).
// FUSED: the operand is p = r + beta p_old (r alone on the first step), p is
// stored and x takes its update for the owned rows; the thread's own p_old
// and x values come with the plane loads, one plane ahead of their use.
// A thread owns kStR = 2 vertically adjacent rows: each one's row sum Sx and
// centre value serve the other's D and Sy from registers.
template <bool ISO, bool FUSED>
__device__ __forceinline__ double stencil_column(const StencilGeom &g, const StencilIO &io, long long t,
                                                 int zlo, int zhi, double *buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = (int)(t % g.ntx), ty = (int)(t / g.ntx);
    const int x0 = 1 + kStX * tx, y0 = 1 + kStY * ty;
    const long long sxy = (long long)(g.nx + 1) * (g.ny + 1);
    const int sr0 = kStR * warp + 1;                  // staged row of the first own node
    const int c0 = sr0 * kStPitch + lane + 1, c1 = c0 + kStPitch;
    const bool has_h = threadIdx.x < kStHalo;
    const int eh = has_h ? halo_elem(threadIdx.x) : 0;
    const StageSlot s0 = stage_slot(g.nx, g.ny, x0, y0, c0);
    const StageSlot s1 = stage_slot(g.nx, g.ny, x0, y0, c1);
    const StageSlot sh = has_h ? stage_slot(g.nx, g.ny, x0, y0, eh) : StageSlot{0, false};
    const bool upd = FUSED && io.pold != nullptr;
    double *sxb = buf + 2 * kStElems;   // Sx of the staged rows

    // raw loads of one plane (operand, or r and p_old), combined when staged
    double ra0 = 0.0, ra1 = 0.0, rh = 0.0, pa0 = 0.0, pa1 = 0.0, ph = 0.0;
    auto fetch = [&](int q) {
        const bool zin = q >= 1 && q < g.nz;
        const long long b = sxy * q;
        ra0 = (zin && s0.ok) ? io.in[b + s0.off] : 0.0;
        ra1 = (zin && s1.ok) ? io.in[b + s1.off] : 0.0;
        rh = (zin && sh.ok) ? io.in[b + sh.off] : 0.0;
        if (upd) {
            pa0 = (zin && s0.ok) ? io.pold[b + s0.off] : 0.0;
            pa1 = (zin && s1.ok) ? io.pold[b + s1.off] : 0.0;
            ph = (zin && sh.ok) ? io.pold[b + sh.off] : 0.0;
        }
    };
    // the row of plane q - 1 from the plane sums of q - 1 and the carried Q's
    auto row_out = [&](const StageSlot &so, int q, double Xm, double Sxm, double Sym, double Dm, double Qm2,
                       double Q, double pm, double xm, double &acc) {
        double yv;
        if constexpr (ISO) yv = fma(g.c[0], Xm, fma(g.c[3], Dm, Qm2 + Q));
        else yv = fma(g.c[3], Dm, fma(g.c[2], Sym, fma(g.c[1], Sxm, fma(g.c[0], Xm, Qm2 + Q))));
        if (so.ok) {
            const long long i = sxy * (q - 1) + so.off;
            io.out[i] = yv;
            if constexpr (FUSED) {
                io.pnew[i] = Xm;
                if (upd) io.x[i] = fma(io.alpha_old, pm, xm);
            }
            acc = fma(Xm, yv, acc);
        }
    };
    auto plane_q = [&](double X, double Sx, double Sy, double D) -> double {
        if constexpr (ISO) return fma(g.c[3], Sx + Sy, g.c[7] * D);
        else return fma(g.c[7], D, fma(g.c[6], Sy, fma(g.c[5], Sx, g.c[4] * X)));
    };
    fetch(zlo - 1);
    // per own row: centre, row sums and carried Q of plane q - 1 (and q - 2)
    double Xm0 = 0.0, Sxm0 = 0.0, Sym0 = 0.0, Dm0 = 0.0, Qa0 = 0.0, Qb0 = 0.0, pm0 = 0.0, xm0 = 0.0;
    double Xm1 = 0.0, Sxm1 = 0.0, Sym1 = 0.0, Dm1 = 0.0, Qa1 = 0.0, Qb1 = 0.0, pm1 = 0.0, xm1 = 0.0;
    double acc = 0.0;
    int par = 0;
    for (int q = zlo - 1; q <= zhi; ++q) {
        double *s = buf + par * kStElems;
        const double X0 = upd ? fma(io.beta, pa0, ra0) : ra0;
        const double X1 = upd ? fma(io.beta, pa1, ra1) : ra1;
        const double pq0 = pa0, pq1 = pa1;
        s[c0] = X0;
        s[c1] = X1;
        if (has_h) s[eh] = upd ? fma(io.beta, ph, rh) : rh;
        __syncthreads();
        double xq0 = 0.0, xq1 = 0.0;
        if (upd && q >= zlo && q < zhi) {
            if (s0.ok) xq0 = io.x[sxy * q + s0.off];
            if (s1.ok) xq1 = io.x[sxy * q + s1.off];
        }
        if (q < zhi) fetch(q + 1);
        // Sx of every staged row (the own rows' in registers, all of them in
        // shared memory): D is Sx of the rows above and below
        const double Sx0 = s[c0 - 1] + s[c0 + 1];
        const double Sx1 = s[c1 - 1] + s[c1 + 1];
        sxb[sr0 * kStX + lane] = Sx0;
        sxb[(sr0 + 1) * kStX + lane] = Sx1;
        if (warp < 2) {
            const int r = warp == 0 ? 0 : kStY + 1;
            sxb[r * kStX + lane] = s[r * kStPitch + lane] + s[r * kStPitch + lane + 2];
        }
        __syncthreads();
        const double D0 = sxb[(sr0 - 1) * kStX + lane] + Sx1;
        const double D1 = Sx0 + sxb[(sr0 + 2) * kStX + lane];
        const double Sy0 = s[c0 - kStPitch] + X1;
        const double Sy1 = X0 + s[c1 + kStPitch];
        const double Q0 = plane_q(X0, Sx0, Sy0, D0);
        const double Q1 = plane_q(X1, Sx1, Sy1, D1);
        if (q > zlo) {
            row_out(s0, q, Xm0, Sxm0, Sym0, Dm0, Qb0, Q0, pm0, xm0, acc);
            row_out(s1, q, Xm1, Sxm1, Sym1, Dm1, Qb1, Q1, pm1, xm1, acc);
        }
        Qb0 = Qa0; Qa0 = Q0; Xm0 = X0; Dm0 = D0; pm0 = pq0; xm0 = xq0;
        Qb1 = Qa1; Qa1 = Q1; Xm1 = X1; Dm1 = D1; pm1 = pq1; xm1 = xq1;
        if constexpr (!ISO) {
            Sxm0 = Sx0; Sym0 = Sy0;
            Sxm1 = Sx1; Sym1 = Sy1;
        }
        par ^= 1;
    }
    __syncthreads();  // the next column stages into buffer 0 again
    return acc;
}

// Boundary rows: out = operand (identity rows); CG pass as stencil_column.
template <bool FUSED>
__device__ __forceinline__ double stencil_bc_rows(const StencilGeom &g, const StencilIO &io) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const bool upd = FUSED && io.pold != nullptr;
    double acc = 0.0;
    for (long long q = tid; q < g.n_bc; q += nth) {
        const long long i = bc_node(g.nx, g.ny, g.nz, q);
        double v = io.in[i];
        if constexpr (FUSED) {
            if (upd) {
                const double po = io.pold[i];
                v = fma(io.beta, po, v);
                io.x[i] = fma(io.alpha_old, po, io.x[i]);
            }
            io.pnew[i] = v;
        }
        io.out[i] = v;
        acc = fma(v, v, acc);
    }
    return acc;
}


// A whole operator pass by this block: its interior segments, then its share
// of the boundary rows.  Returns the thread's partial of operand . result.
template <bool ISO, bool FUSED>
__device__ __forceinline__ double stencil_pass(const StencilGeom &g, const StencilIO &io, double *buf) {
    double acc = 0.0;
    const int nzi = g.nz - 1;
    long long lo, hi;
    block_range(g, blockIdx.x, gridDim.x, &lo, &hi);
    while (lo < hi) {
        const long long t = lo / nzi;
        const int z0 = (int)(lo - t * nzi);
        const long long left = hi - lo;
        const int z1 = (int)((nzi - z0) < left ? nzi : z0 + left);
        acc += stencil_column<ISO, FUSED>(g, io, t, 1 + z0, 1 + z1, buf);
        lo += z1 - z0;
    }
    acc += stencil_bc_rows<FUSED>(g, io);
    return acc;
}

template <bool ISO>
__global__ void __launch_bounds__(kCgThreads, 3) k_stencil_spmv(const StencilGeom g, const double *x, double *y) {
    __shared__ double buf[kStBuf];
    StencilIO io{x, nullptr, nullptr, nullptr, y, 0.0, 0.0};
    (void)stencil_pass<ISO, false>(g, io, buf);
}

// b_i = g_i on boundary rows; elsewhere 0 - sum over boundary neighbours j of
// a(j - i) g_j (zero source term, boundary columns moved to the right side).
__global__ void k_stencil_rhs(const StencilGeom g, const double *__restrict__ gval, double *__restrict__ b) {
    const long long nxn = g.nx + 1, nyn = g.ny + 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.m;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nxn);
        const long long r = i / nxn;
        const int iy = (int)(r % nyn), iz = (int)(r / nyn);
        const bool bnd = ix == 0 || ix == g.nx || iy == 0 || iy == g.ny || iz == 0 || iz == g.nz;
        if (bnd) {
            b[i] = gval[i];
            continue;
        }
        double s = 0.0;
        if (ix == 1 || ix == g.nx - 1 || iy == 1 || iy == g.ny - 1 || iz == 1 || iz == g.nz - 1) {
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                        if (jx == 0 || jx == g.nx || jy == 0 || jy == g.ny || jz == 0 || jz == g.nz) {
                            const int k = (dx != 0) + 2 * (dy != 0) + 4 * (dz != 0);
                            s = fma(g.c[k], gval[jx + nxn * (jy + nyn * (long long)jz)], s);
                        }
                    }
        }
        b[i] = 0.0 - s;
    }
}

struct StencilCgArgs {
    StencilGeom g;
    const double *b;
    double *x, *r, *p0, *p1, *w;
    double *part;            // [2][2 * kCgMaxBlocks]
    CgCtrl *ctrl;
    double tol2;
    int maxit;
    long long timeout_ns;
    long long stall_barrier;
};

template <bool ISO>
__global__ void __launch_bounds__(kCgThreads, 2) k_cg_stencil(const StencilCgArgs a) {
    __shared__ CgBlockState st;
    __shared__ double buf[kStBuf];
    const long long m = a.g.m;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    if (threadIdx.x == 0) {
        st.target = 0;
        st.round = 0;
        st.k = 0;
        st.ok = 1;
    }
    __syncthreads();
    int status = FE_ERR_MAXIT;
    bool alive;
    // r = b - A x: w = A x, then a row pass (another block's rows of w)
    {
        StencilIO io{a.x, nullptr, nullptr, nullptr, a.w, 0.0, 0.0};
        (void)stencil_pass<ISO, false>(a.g, io, buf);
        alive = grid_barrier(a.ctrl, &st, a.timeout_ns, a.stall_barrier);
        double s0 = 0.0, s1 = 0.0;
        if (alive) {
            for (long long i = tid; i < m; i += nth) {
                const double bi = a.b[i], ri = bi - a.w[i];
                a.r[i] = ri;
                s0 = fma(ri, ri, s0);
                s1 = fma(bi, bi, s1);
            }
        }
        double rr0 = 0.0, bb0 = 0.0;
        if (alive) alive = grid_sum2(a, &st, s0, s1, rr0, bb0);
        if (threadIdx.x == 0) {
            st.rr = rr0;
            st.bb = bb0;
        }
        __syncthreads();
    }
    // Step k writes p into p0 (k even) or p1 (k odd) and reads the other one
    // as p_old.  alpha_old and beta live in shared memory, so that only
    // status flags stay in registers across the operator pass.
    __shared__ double coef[2];           // alpha_old, beta
    if (threadIdx.x == 0) coef[0] = coef[1] = 0.0;
    __syncthreads();
    if (alive && st.bb == 0.0) {         // b = 0: the solution is 0
        for (long long i = tid; i < m; i += nth) a.x[i] = 0.0;
        if (threadIdx.x == 0) st.rr = 0.0;
        status = FE_OK;
    } else {
        while (alive) {
            if (st.rr <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
            // A: p = r + beta p_old, x += alpha_old p_old, w = A p, p.w
            const int k = st.k;
            double *pcur = (k & 1) ? a.p1 : a.p0;
            const double *pold = k > 0 ? ((k & 1) ? a.p0 : a.p1) : nullptr;
            const StencilIO io{a.r, pold, pcur, a.x, a.w, coef[1], coef[0]};
            const double pw_part = stencil_pass<ISO, true>(a.g, io, buf);
            double pw, alpha;                // alpha = rr / (p.w), formed once per block
            if (!(alive = grid_sum1_div<1>(a, &st, pw_part, st.rr, pw, alpha))) break;
            if (!(pw > 0.0) || !(pw < INFINITY)) { status = FE_ERR_BREAKDOWN; break; }
            // B: r -= alpha w, r.r
            const double rr_part = update_r<double>(a.r, a.w, a.g.m, alpha);
            double rr_new;
            if (!(alive = grid_sum1(a, &st, rr_part, rr_new))) break;
            __syncthreads();   // every thread has read st.rr and coef
            if (threadIdx.x == 0) {
                coef[0] = alpha;
                coef[1] = rr_new / st.rr;
                st.rr = rr_new;
                st.k += 1;
            }
            __syncthreads();
            if (rr_new <= a.tol2 * st.bb) { status = FE_OK; break; }
            if (st.k >= a.maxit) { status = FE_ERR_MAXIT; break; }
        }
    }
    // the last x update (x lacks alpha_old p of the last step taken), row by row
    if (alive && st.k > 0 && (status == FE_OK || status == FE_ERR_MAXIT)) {
        const double *plast = (st.k & 1) ? a.p0 : a.p1;   // written by step k - 1
        const double al = coef[0];
        for (long long i = tid; i < m; i += nth) a.x[i] = fma(al, plast[i], a.x[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctrl->status = alive ? status : FE_ERR_TIMEOUT;
        a.ctrl->iterations = st.k;
        a.ctrl->rr = st.rr;
        a.ctrl->bb = st.bb;
    }
}

// ---------------------------------------------------------------- host side


static bool stencil_iso(const StencilGeom &g) { return g.nx == g.ny && g.ny == g.nz; }

static size_t align256s(size_t n) { return (n + 255) & ~(size_t)255; }

static size_t stencil_cg_bytes(const StencilGeom &g) {
    const size_t vec = align256s((size_t)g.m * sizeof(double));
    return 256 + align256s(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) + 4 * vec;
}

template <class K> static fe_status stencil_blocks(K kern, int *blocks) {
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCgThreads, 0));
    if (per_sm < 1) return FE_ERR_CUDA;
    long long n = (long long)sm_count() * per_sm;
    if (n > kCgMaxBlocks) n = kCgMaxBlocks;
    *blocks = (int)(n < 1 ? 1 : n);
    return FE_OK;
}

template <bool ISO>
static fe_status launch_stencil_cg(const StencilCgArgs &args, cudaStream_t s) {
    auto kern = k_cg_stencil<ISO>;
    int blocks = 0;
    fe_status st = stencil_blocks(kern, &blocks);
    if (st != FE_OK) return st;
    void *params[] = {(void *)&args};
    FE_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)blocks), dim3(kCgThreads), params,
                                            0, s));
    return FE_OK;
}

template <bool ISO>
static fe_status launch_stencil_spmv(const StencilGeom &g, const double *x, double *y, cudaStream_t s) {
    auto kern = k_stencil_spmv<ISO>;
    int blocks = 0;
    fe_status st = stencil_blocks(kern, &blocks);
    if (st != FE_OK) return st;
    kern<<<blocks, kCgThreads, 0, s>>>(g, x, y);
    FE_TRY_LAUNCH();
    return FE_OK;
}

// sum over rows of (b - y)^2 and b^2, per block
static __global__ void __launch_bounds__(kCgThreads) k_stencil_resid(long long m, const double *__restrict__ b,
                                                                     const double *__restrict__ y,
                                                                     double *__restrict__ part) {
    __shared__ double red[kCgWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s0 = 0.0, s1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const double bi = b[i], ri = bi - y[i];
        s0 = fma(ri, ri, s0);
        s1 = fma(bi, bi, s1);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (lane == 0) {
        red[warp][0] = s0;
        red[warp][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int k = 0; k < kCgWarps; ++k) {
            t0 += red[k][0];
            t1 += red[k][1];
        }
        part[2 * blockIdx.x] = t0;
        part[2 * blockIdx.x + 1] = t1;
    }
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_stencil_spmv(int nx, int ny, int nz, const double *d_x, double *d_y, fe_stream_t stream) {
    StencilGeom g;
    if (!stencil_geom(nx, ny, nz, &g) || !d_x || !d_y) return FE_ERR_ARG;
    if (!aligned(d_x, 8) || !aligned(d_y, 8) || d_x == d_y) return FE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    return stencil_iso(g) ? launch_stencil_spmv<true>(g, d_x, d_y, s) : launch_stencil_spmv<false>(g, d_x, d_y, s);
}

fe_status fe_stencil_rhs(int nx, int ny, int nz, const double *d_bc_val, double *d_b, fe_stream_t stream) {
    StencilGeom g;
    if (!stencil_geom(nx, ny, nz, &g) || !d_bc_val || !d_b) return FE_ERR_ARG;
    if (!aligned(d_bc_val, 8) || !aligned(d_b, 8) || d_bc_val == d_b) return FE_ERR_ARG;
    long long blocks = (g.m + 255) / 256;
    const long long cap = (long long)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    k_stencil_rhs<<<(int)(blocks < 1 ? 1 : blocks), 256, 0, (cudaStream_t)stream>>>(g, d_bc_val, d_b);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_stencil_cg_workspace(int nx, int ny, int nz, size_t *h_bytes) {
    StencilGeom g;
    if (!stencil_geom(nx, ny, nz, &g) || !h_bytes) return FE_ERR_ARG;
    *h_bytes = stencil_cg_bytes(g);
    return FE_OK;
}

fe_status fe_stencil_cg_solve(int nx, int ny, int nz, const double *d_b, double *d_x, double tol, int maxit,
                              double timeout_s, void *d_work, size_t work_bytes, fe_cg_result *h_result,
                              fe_stream_t stream) {
    StencilGeom g;
    if (!stencil_geom(nx, ny, nz, &g)) return FE_ERR_ARG;
    if (!d_b || !d_x || !d_work || !h_result || maxit < 0 || !(tol >= 0.0)) return FE_ERR_ARG;
    if (!aligned(d_b, 8) || !aligned(d_x, 8) || !aligned(d_work, 256)) return FE_ERR_ARG;
    if (work_bytes < stencil_cg_bytes(g)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)d_work;
    StencilCgArgs args;
    args.g = g;
    args.b = d_b;
    args.x = d_x;
    args.ctrl = (CgCtrl *)ws;
    args.part = (double *)(ws + 256);
    const size_t vec = align256s((size_t)g.m * sizeof(double));
    char *v0 = ws + 256 + align256s(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double));
    args.r = (double *)v0;
    args.p0 = (double *)(v0 + vec);
    args.p1 = (double *)(v0 + 2 * vec);
    args.w = (double *)(v0 + 3 * vec);
    args.tol2 = tol * tol;
    args.maxit = maxit;
    const double tmo = timeout_s > 0.0 ? timeout_s : 2.0;
    args.timeout_ns = (long long)(tmo * 1e9);
    args.stall_barrier = take_stall_barrier();
    FE_TRY_CUDA(cudaMemsetAsync(args.ctrl, 0, sizeof(CgCtrl), s));
    fe_status st = stencil_iso(g) ? launch_stencil_cg<true>(args, s) : launch_stencil_cg<false>(args, s);
    if (st != FE_OK) return st;
    CgCtrl ctrl;
    FE_TRY_CUDA(cudaMemcpyAsync(&ctrl, args.ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    h_result->status = ctrl.status;
    h_result->iterations = ctrl.iterations;
    h_result->bnorm = sqrt(ctrl.bb);
    h_result->relres = ctrl.bb > 0.0 ? sqrt(ctrl.rr / ctrl.bb) : 0.0;
    return (fe_status)ctrl.status;
}

fe_status fe_stencil_true_relres(int nx, int ny, int nz, const double *d_b, const double *d_x, void *d_work,
                                 size_t work_bytes, double *h_relres, fe_stream_t stream) {
    StencilGeom g;
    if (!stencil_geom(nx, ny, nz, &g)) return FE_ERR_ARG;
    if (!d_b || !d_x || !d_work || !h_relres) return FE_ERR_ARG;
    if (!aligned(d_b, 8) || !aligned(d_x, 8) || !aligned(d_work, 256)) return FE_ERR_ARG;
    if (work_bytes < stencil_cg_bytes(g)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)d_work;
    double *part = (double *)(ws + 256);
    double *out = part + 2 * kCgMaxBlocks;
    const size_t vec = align256s((size_t)g.m * sizeof(double));
    double *y = (double *)(ws + 256 + align256s(2 * 2 * (size_t)kCgMaxBlocks * sizeof(double)) + 3 * vec);
    fe_status st = stencil_iso(g) ? launch_stencil_spmv<true>(g, d_x, y, s) : launch_stencil_spmv<false>(g, d_x, y, s);
    if (st != FE_OK) return st;
    long long blocks = (long long)sm_count() * 4;
    const long long need = (g.m + kCgThreads - 1) / kCgThreads;
    if (blocks > need) blocks = need;
    if (blocks > kCgMaxBlocks) blocks = kCgMaxBlocks;
    if (blocks < 1) blocks = 1;
    k_stencil_resid<<<(int)blocks, kCgThreads, 0, s>>>(g.m, d_b, y, part);
    FE_TRY_LAUNCH();
    k_resid_final<<<1, 32, 0, s>>>((int)blocks, part, out);
    FE_TRY_LAUNCH();
    double h[2];
    FE_TRY_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    FE_TRY_CUDA(cudaStreamSynchronize(s));
    *h_relres = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
    return FE_OK;
}

}  // extern "C"
