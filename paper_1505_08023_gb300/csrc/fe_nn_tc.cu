// fe_nn_tc.cu -- the 3x3x3 convolutions of the warm-start network (stride 1,
// stride 2, transposed stride 2) on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory).
//
// out[co][u] = bias[co] + sum_ci sum_t W[ci][t][co] in[ci][u + d_t - 1]  (tap t = 9dz + 3dy + dx)
//
// As a GEMM: D[u][co] = sum_k A[u][k] B[co][k] with k = (ci, t).  No im2col
// copy is made.  A block owns TY output lines of one z-plane; for each chunk
// of 16 input channels it stages the halo box (3 planes x (TY + 2) lines x
// (W + 2) points) in shared memory as rows of 16 bytes (one voxel, 8 BF16
// channels), two 8-channel groups one after the other.  In that layout the
// operand A of tap t is the same matrix shifted by a whole number of rows,
// shift(t) = (dz - 1)(TY + 2)(W + 2) + (dy - 1)(W + 2) + (dx - 1), so every
// tap is one tcgen05.mma whose A descriptor starts shift(t) rows further.
// The output rows of the tile are a contiguous run of halo rows (the halo
// columns between lines are computed and dropped), covered by nw windows of
// 128 rows (M = 128).  B (the chunk's weights, N = cout) is a pre-packed
// image copied as is.  One thread issues the nw x 27 MMAs of a chunk and
// commits them to an mbarrier; the FP32 accumulators of the nw windows live
// in tensor memory until the epilogue reads them (tcgen05.ld), adds the bias,
// applies ReLU and writes FP32 [C][D][H][W].
//
// Operands: activations rounded to BF16 (nearest even), weights BF16, FP32
// accumulation.  Shared-memory matrix layout: no swizzle, K-major core
// matrices of 8 rows x 16 bytes; leading offset = distance between the two
// 8-channel groups, stride offset = 128 bytes (rows are contiguous).
// Every wait is bounded; a block that gives up sets the error flag read by
// fe_nn_tc_check, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "fe_common.cuh"

namespace fe {

constexpr int kTcThreads = 256;
constexpr int kTcMaxTY = 8;
constexpr size_t kTcSmemCap = 200 * 1024;

static __device__ int g_tc_err;

struct TcDims {
    int d, h, w;
};

// Tile geometry (host-chosen): TY output lines per tile, W2 = W + 2 halo row
// length, rows = staged halo rows, rows_pad = rows incl. the zero rows the
// last window may read, base = halo row of output (y0, x 0), nw = windows.
struct TcGeom {
    int ty, w2, rows, rows_pad, base, nw, tmem_cols, ctas_per_sm;
    int hlo, ly, pz;   // halo below the tile (1: stride 1, 0: transposed), lines and planes staged
    int rsub;          // stride 2: rows of one of the eight parity sub-boxes
    int tma_rows;      // rows one 8-channel group's box loads write (TMA staging)
    size_t smem;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ long long tc_now() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up (1 s).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const long long t0 = tc_now();
    for (unsigned it = 0; it < (1u << 26); ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && tc_now() - t0 > 1000000000LL) return false;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Stride 2 (FE_NN_S2) stages the fine input box as eight parity sub-boxes
// on the coarse output lattice, so that each tap again reads one sub-box at
// a uniform shift.
// MODE = FE_NN_S1 (one class, all 27 taps, dout = din) or FE_NN_T2 (the
// transposed stride-2 layer: eight output parity classes p, output 2v + p of
// input position v; per axis p = 0 takes tap d = 1 at offset 0, p = 1 takes
// d = 0 at offset +1 and d = 2 at offset 0 -- 27 (class, tap) pairs in all,
// each an MMA on the input box shifted by its offsets; class c accumulates
// in its own tensor-memory columns).
//
// TMA = true: the input comes as BF16 in the 8-channel-interleaved layout
// [ceil(C/8)][D][H][W][8] (fe_nn_to_bf16i) and one thread stages each chunk
// with tensor-map box loads (cp.async.bulk.tensor, zero fill outside the
// grid; element stride 2 for the parity sub-boxes of the stride-2 layer) and
// the chunk's weights with one bulk copy, all completing on an mbarrier.
// TMA = false: every thread loads FP32 [C][D][H][W] and converts.
template <int MODE, bool TMA>
__global__ void __launch_bounds__(kTcThreads, 1)
k_conv_tc(const float *__restrict__ in, int cin, TcDims dm, const __nv_bfloat16 *__restrict__ wimg,
          const float *__restrict__ bias, float *__restrict__ out, int cout, TcDims dout, int relu, TcGeom g,
          const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t mbar_ld;   // TMA staging
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    __shared__ uint64_t s_adesc[27], s_bdesc[27];   // per (class, tap) operand descriptors, window 0
    __shared__ int s_col[27];                       // tensor-memory column of the entry's class
    __shared__ int s_first[27];                     // 1 for the first entry of a class
    unsigned char *sA = smem;                                  // [2][rows_pad][8] bf16
    unsigned char *sB = smem + (size_t)2 * g.rows_pad * 16;    // [27][2][cout][8] bf16
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = dm.w, H = dm.h, D = dm.d, W2 = g.w2, TY = g.ty, LY = g.ly, HLO = g.hlo;
    const size_t plane = (size_t)D * H * W;
    const size_t oplane = (size_t)dout.d * dout.h * dout.w;
    // tiles run over the grid whose positions the MMA rows stand for: the
    // output grid for stride 2, the input grid otherwise
    const int TD = MODE == FE_NN_S2 ? dout.d : D, TH = MODE == FE_NN_S2 ? dout.h : H;
    const int TW = MODE == FE_NN_S2 ? dout.w : W;
    const int nty = (TH + TY - 1) / TY;
    const int ntiles = TD * nty;
    const int nkc = (cin + 15) / 16;
    const size_t chunk_bytes = (size_t)27 * 2 * cout * 16;
    const uint32_t mbar_a = smem_u32(&mbar);

    if (tid == 0) {
        int e = 0;
        const int ncls = MODE == FE_NN_T2 ? 8 : 1;
        for (int c = 0; c < ncls; ++c) {
            const int pz = (c >> 2) & 1, py = (c >> 1) & 1, px = c & 1;
            const int nz = MODE == FE_NN_T2 ? (pz ? 2 : 1) : 3;
            const int ny = MODE == FE_NN_T2 ? (py ? 2 : 1) : 3;
            const int nx = MODE == FE_NN_T2 ? (px ? 2 : 1) : 3;
            for (int iz = 0; iz < nz; ++iz)
                for (int iy = 0; iy < ny; ++iy)
                    for (int ix = 0; ix < nx; ++ix) {
                        int dz, dy, dx, oz, oy, ox, sub = 0;
                        if (MODE == FE_NN_S2) {
                            // fine input 2v + d - 1: d = 1 is the even point v,
                            // d = 0 the odd point v - 1, d = 2 the odd point v
                            dz = iz; dy = iy; dx = ix;
                            oz = iz == 0 ? -1 : 0; oy = iy == 0 ? -1 : 0; ox = ix == 0 ? -1 : 0;
                            sub = ((iz != 1) << 2) | ((iy != 1) << 1) | (ix != 1);
                        } else if (MODE == FE_NN_T2) {
                            dz = pz ? 2 * iz : 1; oz = pz ? 1 - iz : 0;
                            dy = py ? 2 * iy : 1; oy = py ? 1 - iy : 0;
                            dx = px ? 2 * ix : 1; ox = px ? 1 - ix : 0;
                        } else {
                            dz = iz; dy = iy; dx = ix;
                            oz = iz - 1; oy = iy - 1; ox = ix - 1;
                        }
                        const int t = 9 * dz + 3 * dy + dx;
                        const int shift = sub * g.rsub + oz * LY * W2 + oy * W2 + ox;
                        s_adesc[e] = umma_smem_desc(smem_u32(sA) + (uint32_t)(g.base + shift) * 16,
                                                    (uint32_t)g.rows_pad * 16, 128);
                        s_bdesc[e] = umma_smem_desc(smem_u32(sB) + (uint32_t)(t * 2 * cout * 16), (uint32_t)cout * 16, 128);
                        s_col[e] = c * g.nw * cout;
                        s_first[e] = (iz == 0 && iy == 0 && ix == 0) ? 1 : 0;
                        ++e;
                    }
        }
    }
    if (tid == 0) {
        s_ok = 1;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_a), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar_ld)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (TMA) {
        // rows the box loads never write (padding, sub-box gaps) stay zero
        for (size_t i = tid; i < (size_t)2 * g.rows_pad; i += kTcThreads)
            reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = umma_idesc_bf16(128, cout);
    uint32_t phase = 0, ld_phase = 0;
    bool ok = true;

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int z = tile / nty, y0 = (tile % nty) * TY;
        for (int kc = 0; kc < nkc && ok; ++kc) {
            if (TMA) {
                // one thread issues the chunk's box loads and the weight copy
                if (tid == 0) {
                    const uint32_t mb = smem_u32(&mbar_ld);
                    const uint32_t tx = (uint32_t)(2 * g.tma_rows * 16) + (uint32_t)chunk_bytes;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx) : "memory");
                    const uint64_t tm = reinterpret_cast<uint64_t>(&tmap);
                    for (int kg = 0; kg < 2; ++kg) {
                        const int grp = 2 * kc + kg;
                        const int nsub = MODE == FE_NN_S2 ? 8 : 1;
                        for (int sb = 0; sb < nsub; ++sb) {
                            int cx, cy, cz;
                            if (MODE == FE_NN_S2) {
                                cx = -2 + (sb & 1);
                                cy = 2 * (y0 - 1) + ((sb >> 1) & 1);
                                cz = 2 * (z - 1) + ((sb >> 2) & 1);
                            } else {
                                cx = -HLO;
                                cy = y0 - HLO;
                                cz = z - HLO;
                            }
                            const uint32_t dst = smem_u32(sA) + (uint32_t)(((size_t)kg * g.rows_pad + (size_t)sb * g.rsub) * 16);
                            asm volatile(
                                "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes "
                                "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
                                "l"(tm), "r"(0), "r"(cx), "r"(cy), "r"(cz), "r"(grp), "r"(mb)
                                : "memory");
                        }
                    }
                    const unsigned char *src = reinterpret_cast<const unsigned char *>(wimg) + (size_t)kc * chunk_bytes;
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 ::"r"(smem_u32(sB)), "l"(src), "r"((uint32_t)chunk_bytes), "r"(mb) : "memory");
                }
                if (!mbar_wait(smem_u32(&mbar_ld), ld_phase & 1u)) {
                    atomicExch(&g_tc_err, 1);
                    s_ok = 0;
                }
                ld_phase += 1;
            } else {
                // stage the halo box of channels kc*16 .. kc*16+15 (zero outside the
                // grid): four rows per thread per trip, all 64 loads issued first
                for (int r0 = tid; r0 < g.rows_pad; r0 += 4 * kTcThreads) {
                    float v[4][16];
    #pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = r0 + i * kTcThreads;
                        bool inb = false;
                        size_t gidx = 0;
                        if (r < g.rows) {
                            int gz, gy, gx;
                            if (MODE == FE_NN_S2) {
                                // parity sub-box s holds the fine points 2c + parity(s)
                                // of coarse positions c = tile origin - 1 + (a, b, x)
                                const int sb = r / g.rsub, rr = r % g.rsub;
                                const int a = rr / (LY * W2), rem = rr % (LY * W2);
                                const int b = rem / W2, xx = rem % W2;
                                gz = 2 * (z - 1 + a) + ((sb >> 2) & 1);
                                gy = 2 * (y0 - 1 + b) + ((sb >> 1) & 1);
                                gx = 2 * (xx - 1) + (sb & 1);
                            } else {
                                const int pz = r / (LY * W2), rem = r % (LY * W2);
                                const int ly = rem / W2, lx = rem % W2;
                                gz = z - HLO + pz;
                                gy = y0 - HLO + ly;
                                gx = lx - HLO;
                            }
                            inb = gz >= 0 && gz < D && gy >= 0 && gy < H && gx >= 0 && gx < W;
                            gidx = inb ? ((size_t)gz * H + gy) * W + gx : 0;
                        }
    #pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const int ch = kc * 16 + c;
                            v[i][c] = (inb && ch < cin) ? in[(size_t)ch * plane + gidx] : 0.0f;
                        }
                    }
    #pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = r0 + i * kTcThreads;
                        if (r >= g.rows_pad) break;
    #pragma unroll
                        for (int kg = 0; kg < 2; ++kg) {
                            __nv_bfloat162 h[4];
    #pragma unroll
                            for (int j = 0; j < 4; ++j)
                                h[j] = __floats2bfloat162_rn(v[i][8 * kg + 2 * j], v[i][8 * kg + 2 * j + 1]);
                            *reinterpret_cast<uint4 *>(sA + ((size_t)kg * g.rows_pad + r) * 16) =
                                *reinterpret_cast<const uint4 *>(h);
                        }
                    }
                }
                // the chunk's weight image
                const uint4 *src = reinterpret_cast<const uint4 *>(
                    reinterpret_cast<const unsigned char *>(wimg) + (size_t)kc * chunk_bytes);
                for (size_t i = tid; i < chunk_bytes / 16; i += kTcThreads)
                    reinterpret_cast<uint4 *>(sB)[i] = src[i];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // descriptors advance by one unit per 16-byte row: window w, tap t
                // is the window-0 descriptor of t plus 128 w (no field overflows:
                // shared addresses stay below 256 KB)
                for (int e = 0; e < 27; ++e) {
                    const uint32_t acc = (kc > 0 || !s_first[e]) ? 1u : 0u;
                    const uint64_t db = s_bdesc[e];
                    for (int w = 0; w < g.nw; ++w) {
                        const uint32_t d_tmem = tmem + (uint32_t)(s_col[e] + w * cout);
                        const uint64_t da = s_adesc[e] + (uint64_t)(128 * w);
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                                     "l"(da), "l"(db), "r"(idesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 mbar_a)
                             : "memory");
            }
            // the MMAs have read the staged chunk (and written D) once this phase completes
            if (!mbar_wait(mbar_a, phase & 1u)) {
                atomicExch(&g_tc_err, 1);
                s_ok = 0;
            }
            phase += 1;
            __syncthreads();
            ok = s_ok != 0;
        }
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp q (mod 4) reads TMEM lanes 32q..32q+31; the two warpgroups split the columns
        const int q = warp & 3, half = warp >> 2;
        const int c_lo = half * (cout / 2), c_hi = c_lo + cout / 2;
        const int ncls = MODE == FE_NN_T2 ? 8 : 1;
        for (int cls = 0; cls < ncls; ++cls) {
            const int pz = (cls >> 2) & 1, py = (cls >> 1) & 1, px = cls & 1;
            for (int w = 0; w < g.nw; ++w) {
                const int rel = 128 * w + 32 * q + lane;      // row offset from `base`
                const int yi = rel / W2, x = rel % W2;
                const int y = y0 + yi;
                bool valid = x < TW && yi < TY && y < TH;
                int oz = z, oy = y, ox = x;                    // output position
                if (MODE == FE_NN_T2) {
                    oz = 2 * z + pz;
                    oy = 2 * y + py;
                    ox = 2 * x + px;
                    valid = valid && oz < dout.d && oy < dout.h && ox < dout.w;
                }
                const size_t o = ((size_t)oz * dout.h + oy) * dout.w + ox;
                for (int c0 = c_lo; c0 < c_hi; c0 += 8) {
                    float v[8];
                    tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((cls * g.nw + w) * cout + c0), v);
                    if (valid) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float y_ = v[j] + (bias ? bias[c0 + j] : 0.0f);
                            if (relu) y_ = y_ > 0.0f ? y_ : 0.0f;
                            out[(size_t)(c0 + j) * oplane + o] = y_;
                        }
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
}

// image[kc][t][kg][n][c] = W[ci = 16 kc + 8 kg + c][t][n] (0 past cin), from
// the BF16 weights [cin][27][cout].
__global__ void k_pack_mma(const __nv_bfloat16 *__restrict__ w16, int cin, int cout,
                           __nv_bfloat16 *__restrict__ img, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % 8);
        size_t r = i / 8;
        const int nn = (int)(r % cout);
        r /= cout;
        const int kg = (int)(r % 2);
        r /= 2;
        const int t = (int)(r % 27);
        const int kc = (int)(r / 27);
        const int ci = 16 * kc + 8 * kg + c;
        img[i] = ci < cin ? w16[((size_t)ci * 27 + t) * cout + nn] : __float2bfloat16(0.0f);
    }
}

static int pow2_at_least(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

// Tile height TY for a W-wide input grid: the largest share of useful rows
// in the 128-row windows, among the shapes whose shared memory and tensor
// memory fit.  Stride 1 stages a halo of one point on each side; the
// transposed layer only reads offsets 0 and +1, so its box starts at the tile.
static bool choose_geom(int mode, int w, int h, int cout, TcGeom *out, bool tma = false) {
    bool found = false;
    double best = -1.0;
    const int classes = mode == FE_NN_T2 ? 8 : 1;
    for (int ty = 1; ty <= kTcMaxTY && ty <= h; ++ty) {
        TcGeom g;
        g.ty = ty;
        int shift_max;
        if (mode == FE_NN_S2) {
            // eight parity sub-boxes, each 2 planes x (TY + 1) lines x (W + 1)
            // coarse positions starting one before the tile
            g.hlo = 1;
            g.ly = ty + 1;
            g.pz = 2;
            g.w2 = w + 1;
            g.rsub = (g.pz * g.ly * g.w2 + 7) & ~7;   // sub-box regions start on 128-byte boundaries
            g.rows = 8 * g.rsub;
            g.tma_rows = 8 * g.pz * g.ly * g.w2;
            g.base = g.ly * g.w2 + g.w2 + 1;
            shift_max = 7 * g.rsub;
        } else {
            g.hlo = mode == FE_NN_S1 ? 1 : 0;
            g.ly = ty + 1 + g.hlo;
            g.pz = 2 + g.hlo;
            g.w2 = w + 1 + g.hlo;
            g.rows = g.pz * g.ly * g.w2;
            g.rsub = g.rows;
            g.tma_rows = g.rows;
            g.base = g.hlo * (g.ly * g.w2 + g.w2 + 1);
            shift_max = g.ly * g.w2 + g.w2 + 1;
        }
        g.nw = ((ty - 1) * g.w2 + w + 127) / 128;
        const int need = g.base + 128 * g.nw + shift_max;
        g.rows_pad = ((need > g.rows ? need : g.rows) + 7) & ~7;
        g.smem = (size_t)2 * g.rows_pad * 16 + (size_t)27 * 2 * cout * 16;
        g.tmem_cols = pow2_at_least(classes * g.nw * cout);
        if (g.smem > kTcSmemCap || g.tmem_cols > 512) continue;
        if (tma) {   // box dimensions (elements traversed) are at most 256
            const int bx = mode == FE_NN_S2 ? 2 * g.w2 : g.w2, by = mode == FE_NN_S2 ? 2 * g.ly : g.ly;
            if (bx > 256 || by > 256) continue;
        }
        int by_smem = (int)((227 * 1024) / (g.smem + 1024));
        int by_tmem = 512 / g.tmem_cols;
        g.ctas_per_sm = by_smem < by_tmem ? by_smem : by_tmem;
        if (g.ctas_per_sm < 1) continue;
        const double eff = (double)ty * w / (g.nw * 128.0) * (g.ctas_per_sm >= 2 ? 1.0 : 0.85);
        if (eff > best + 1e-9) {
            best = eff;
            *out = g;
            found = true;
        }
    }
    return found;
}

typedef CUresult (*TensorMapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up once)
static TensorMapEncodeFn tensor_map_encoder() {
    static std::once_flag once;
    static TensorMapEncodeFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (TensorMapEncodeFn)p;
    });
    return fn;
}

// Tensor map of a BF16 8-channel-interleaved volume [G][D][H][W][8] whose
// box is pz planes x ly lines x w2 points (elements traversed, so twice that
// with element stride 2 on the spatial axes for the stride-2 parity sub-boxes).
static bool encode_box_map(CUtensorMap *tm, bool s2, const void *d_in16, int c, const int *dims, int w2, int ly,
                           int pz) {
    TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t W = (cuuint64_t)dims[2], H = (cuuint64_t)dims[1], D = (cuuint64_t)dims[0];
    const cuuint64_t G = (cuuint64_t)((c + 7) / 8);
    const cuuint64_t gdim[5] = {8, W, H, D, G};
    const cuuint64_t gstr[4] = {16, 16 * W, 16 * W * H, 16 * W * H * D};
    const cuuint32_t box[5] = {8, (cuuint32_t)(s2 ? 2 * w2 : w2), (cuuint32_t)(s2 ? 2 * ly : ly),
                               (cuuint32_t)(s2 ? 2 * pz : pz), 1};
    const cuuint32_t es[5] = {1, s2 ? 2u : 1u, s2 ? 2u : 1u, s2 ? 2u : 1u, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(d_in16), gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool encode_input_map(CUtensorMap *tm, int mode, const void *d_in16, int cin, const int *dims,
                             const TcGeom &g) {
    return encode_box_map(tm, mode == FE_NN_S2, d_in16, cin, dims, g.w2, g.ly, g.pz);
}

template <int MODE, bool TMA>
static fe_status launch_tc(const float *d_in, const void *d_in16, int cin, const int *h_dims, const void *d_img,
                           const float *d_bias, float *d_out, int cout, const int *h_dims_out, int relu,
                           cudaStream_t stream) {
    if (cout != 16 && cout != 32 && cout != 64) return FE_ERR_ARG;
    if (!aligned(d_img, 16)) return FE_ERR_ARG;
    // the MMA rows stand for output positions (stride 2) or input positions
    const int *tdims = MODE == FE_NN_S2 ? h_dims_out : h_dims;
    TcGeom g;
    if (!choose_geom(MODE, tdims[2], tdims[1], cout, &g, TMA)) return FE_ERR_ARG;
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    if (TMA && !encode_input_map(&tm, MODE, d_in16, cin, h_dims, g)) return FE_ERR_CUDA;
    // request enough shared memory that no more than ctas_per_sm blocks share
    // an SM, so their tensor-memory allocations always fit together
    size_t smem = g.smem;
    const size_t floor_bytes = (size_t)233472 / (size_t)(g.ctas_per_sm + 1) - 1024 + 16;
    if (smem < floor_bytes) smem = floor_bytes;
    if (smem > (size_t)232448) smem = 232448;
    auto kern = k_conv_tc<MODE, TMA>;
    FE_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FE_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    FE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcThreads, smem));
    if (per_sm < 1) return FE_ERR_CUDA;
    if (per_sm > g.ctas_per_sm) return FE_ERR_CUDA;       // tensor memory would be oversubscribed
    const long long ntiles = (long long)tdims[0] * ((tdims[1] + g.ty - 1) / g.ty);
    // ctas_per_sm blocks per SM (shared and tensor memory admit them; the
    // occupancy query answers 1 for this kernel although the SM holds 2): a
    // second CTA's staging and MMAs overlap the first's epilogue.  The tiles
    // are independent, so blocks that do not fit simply run later.
    long long grid = (long long)sm_count() * g.ctas_per_sm;
    if (grid > ntiles) grid = ntiles;
    TcDims dm{h_dims[0], h_dims[1], h_dims[2]};
    TcDims dout{h_dims_out[0], h_dims_out[1], h_dims_out[2]};
    kern<<<(int)grid, kTcThreads, smem, stream>>>(d_in, cin, dm, (const __nv_bfloat16 *)d_img, d_bias, d_out,
                                                   cout, dout, relu, g, tm);
    FE_TRY_LAUNCH();
    return FE_OK;
}

// FP32 [C][V] -> BF16 [ceil(C/8)][V][8] (channels past C are 0)
__global__ void k_to_bf16i(const float *__restrict__ in, int c, size_t v, __nv_bfloat16 *__restrict__ out) {
    const int groups = (c + 7) / 8;
    const size_t n = (size_t)groups * v;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int gq = (int)(i / v);
        const size_t vi = i % v;
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c0 = 8 * gq + 2 * j;
            const float a = c0 < c ? in[(size_t)c0 * v + vi] : 0.0f;
            const float b = c0 + 1 < c ? in[(size_t)(c0 + 1) * v + vi] : 0.0f;
            h[j] = __floats2bfloat162_rn(a, b);
        }
        reinterpret_cast<uint4 *>(out)[i] = *reinterpret_cast<const uint4 *>(h);
    }
}

// ---------------------------------------------------------------- weight gradient
//
// R[a][b][t] = sum_z A[a][z] B[b][S z + d_t - 1] over the positions z of A's
// grid (S = 1: the stride-1 layer, A = dY, B = X; S = 2: the stride-2 layer,
// A = dY, B = X, and the transposed layer, A = X, B = dY), on the tensor
// cores.  Per tap t it is a GEMM with the positions as the contraction:
// D_t[a][b] = sum_k A[a][k] B_t[k][b], M = a (padded to 128 rows), N = b,
// K = the tile's positions.  B_t is staged exactly like the forward layer's
// input box (halo box, or eight parity sub-boxes for S = 2) as 16-byte rows of
// one position x 8 channels, so that B_t is the same operand shifted by a
// whole number of rows; read with K along the rows and N along the channels,
// both operands are MN-major (no swizzle: core matrices of 8 positions x 8
// channels, 128 contiguous bytes; the leading offset steps along K, 128
// bytes, the stride offset between 8-channel groups).  A block takes a range
// of tiles (TY lines of one plane) and one group of taps whose accumulators
// fit tensor memory (27 x b columns do not for b > 16), accumulates over its
// tiles and writes its partial R; k_corr_reduce sums the partials in a fixed
// order.  BF16 operands (nearest even), FP32 accumulation.
struct WgGeom {
    int ty, w2, ly, pz, rsub, rows, rows_pad, base, nk;
    int taps_per_group, n_groups, tmem_cols;
    size_t smem;
};

//
// TMA = true: B comes as BF16 in the 8-channel-interleaved layout (a copy in
// the workspace) and thread 0 stages each tile's box with tensor-map box loads
// issued before the threads stage A, so the two overlap; the box is the
// forward layer's (halo box, or the eight parity sub-boxes with element
// stride 2), zero filled outside the grid.  TMA = false: every thread loads
// FP32 B and converts (grids too wide for a 256-point box).
template <int S, bool TMA>
__global__ void __launch_bounds__(kTcThreads, 1)
k_wgrad_tc(const float *__restrict__ A, int ca, TcDims da, const float *__restrict__ B, int cb, TcDims db,
           float *__restrict__ part, WgGeom g, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t mbar_b;     // TMA staging of B
    __shared__ uint32_t tmem_base;
    __shared__ int s_shift[27];
    unsigned char *sA = smem;                                   // [16][nk] rows of 16 bytes
    unsigned char *sB = smem + (size_t)16 * g.nk * 16;          // [cb/8][rows_pad] rows of 16 bytes
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W2 = g.w2, TY = g.ty, LY = g.ly;
    const size_t plane_a = (size_t)da.d * da.h * da.w, plane_b = (size_t)db.d * db.h * db.w;
    const int nty = (da.h + TY - 1) / TY, ntiles = da.d * nty;
    const int t0 = blockIdx.y * g.taps_per_group;
    const int t1 = t0 + g.taps_per_group < 27 ? t0 + g.taps_per_group : 27;
    const int ga = (ca + 7) / 8, gb = cb / 8;
    const uint32_t mbar_a = smem_u32(&mbar);
    if (tid < 27) {
        const int iz = tid / 9, iy = (tid / 3) % 3, ix = tid % 3;
        int shift;
        if (S == 2) {
            const int sub = ((iz != 1) << 2) | ((iy != 1) << 1) | (ix != 1);
            shift = sub * g.rsub + (iz == 0 ? -1 : 0) * LY * W2 + (iy == 0 ? -1 : 0) * W2 + (ix == 0 ? -1 : 0);
        } else {
            shift = (iz - 1) * LY * W2 + (iy - 1) * W2 + (ix - 1);
        }
        s_shift[tid] = shift;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_a), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar_b)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // A's channel groups past ca and every row stay zero unless staged
    for (size_t i = tid; i < (size_t)16 * g.nk; i += kTcThreads)
        reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (TMA) {
        // B rows the box loads never write (padding, sub-box gaps) stay zero
        for (size_t i = tid; i < (size_t)gb * g.rows_pad; i += kTcThreads)
            reinterpret_cast<uint4 *>(sB)[i] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // both operands MN-major (transpose bits of the instruction descriptor)
    const uint32_t idesc = umma_idesc_bf16(128, cb) | (1u << 15) | (1u << 16);
    uint32_t phase = 0, phase_b = 0;
    bool ok = true, first = true, b_pending = false;

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int z = tile / nty, y0 = (tile % nty) * TY;
        if (TMA && tid == 0) {
            // B's box, one load per 8-channel group (and parity sub-box), on mbar_b;
            // the previous tile's MMAs, which read sB, completed before this trip
            const uint32_t mb = smem_u32(&mbar_b);
            const int nsub = S == 2 ? 8 : 1;
            const uint32_t tx = (uint32_t)(gb * nsub * g.pz * LY * W2 * 16);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx) : "memory");
            const uint64_t tm = reinterpret_cast<uint64_t>(&tmap);
            for (int q = 0; q < gb; ++q)
                for (int sb = 0; sb < nsub; ++sb) {
                    int cx, cy, cz;
                    if (S == 2) {
                        cx = -2 + (sb & 1);
                        cy = 2 * (y0 - 1) + ((sb >> 1) & 1);
                        cz = 2 * (z - 1) + ((sb >> 2) & 1);
                    } else {
                        cx = -1;
                        cy = y0 - 1;
                        cz = z - 1;
                    }
                    const uint32_t dst = smem_u32(sB) + (uint32_t)(((size_t)q * g.rows_pad + (size_t)sb * g.rsub) * 16);
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes "
                        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
                        "l"(tm), "r"(0), "r"(cx), "r"(cy), "r"(cz), "r"(q), "r"(mb)
                        : "memory");
                }
        }
        if (TMA) b_pending = true;
        // A over the tile's positions: row j = (line j / W2, point j % W2);
        // the points past the line's end (the box's halo columns) are zero
        for (int j = tid; j < g.nk; j += kTcThreads) {
            const int yi = j / W2, x = j % W2, y = y0 + yi;
            const bool inb = j < TY * W2 && x < da.w && y < da.h;
            const size_t gidx = inb ? ((size_t)z * da.h + y) * da.w + x : 0;
            for (int q = 0; q < ga; ++q) {
                __nv_bfloat162 h[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int c0 = 8 * q + 2 * c;
                    const float v0 = (inb && c0 < ca) ? A[(size_t)c0 * plane_a + gidx] : 0.0f;
                    const float v1 = (inb && c0 + 1 < ca) ? A[(size_t)(c0 + 1) * plane_a + gidx] : 0.0f;
                    h[c] = __floats2bfloat162_rn(v0, v1);
                }
                *reinterpret_cast<uint4 *>(sA + ((size_t)q * g.nk + j) * 16) = *reinterpret_cast<const uint4 *>(h);
            }
        }
        // B's box (zero outside the grid and in the padding rows)
        for (int r = tid; r < (TMA ? 0 : g.rows_pad); r += kTcThreads) {
            bool inb = false;
            size_t gidx = 0;
            if (r < g.rows) {
                int gz, gy, gx;
                if (S == 2) {
                    const int sb = r / g.rsub, rr = r % g.rsub;
                    const int a_ = rr / (LY * W2), rem = rr % (LY * W2);
                    const int b_ = rem / W2, xx = rem % W2;
                    gz = 2 * (z - 1 + a_) + ((sb >> 2) & 1);
                    gy = 2 * (y0 - 1 + b_) + ((sb >> 1) & 1);
                    gx = 2 * (xx - 1) + (sb & 1);
                    inb = rr < g.pz * LY * W2;
                } else {
                    const int pz = r / (LY * W2), rem = r % (LY * W2);
                    gz = z - 1 + pz;
                    gy = y0 - 1 + rem / W2;
                    gx = rem % W2 - 1;
                    inb = true;
                }
                inb = inb && gz >= 0 && gz < db.d && gy >= 0 && gy < db.h && gx >= 0 && gx < db.w;
                gidx = inb ? ((size_t)gz * db.h + gy) * db.w + gx : 0;
            }
            for (int q = 0; q < gb; ++q) {
                __nv_bfloat162 h[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int c0 = 8 * q + 2 * c;
                    const float v0 = inb ? B[(size_t)c0 * plane_b + gidx] : 0.0f;
                    const float v1 = inb ? B[(size_t)(c0 + 1) * plane_b + gidx] : 0.0f;
                    h[c] = __floats2bfloat162_rn(v0, v1);
                }
                *reinterpret_cast<uint4 *>(sB + ((size_t)q * g.rows_pad + r) * 16) = *reinterpret_cast<const uint4 *>(h);
            }
        }
        bool bfail = false;
        if (TMA) {
            if (mbar_wait(smem_u32(&mbar_b), phase_b & 1u)) {
                b_pending = false;
            } else {
                atomicExch(&g_tc_err, 1);
                bfail = true;
            }
            phase_b += 1;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(bfail)) {   // every thread takes the same branch
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int t = t0; t < t1; ++t) {
                const uint32_t d_tmem = tmem + (uint32_t)((t - t0) * cb);
                const uint32_t brow = (uint32_t)(g.base + s_shift[t]);
                for (int kk = 0; kk < g.nk / 16; ++kk) {
                    const uint64_t da_ = umma_smem_desc(a0 + (uint32_t)(kk * 16 * 16), 128u, (uint32_t)g.nk * 16);
                    const uint64_t db_ = umma_smem_desc(b0 + (brow + (uint32_t)(16 * kk)) * 16, 128u,
                                                        (uint32_t)g.rows_pad * 16);
                    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                                 "l"(da_), "l"(db_), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                         : "memory");
        }
        const bool mfail = !mbar_wait(mbar_a, phase & 1u);
        if (mfail) atomicExch(&g_tc_err, 1);
        phase += 1;
        first = false;
        ok = !__syncthreads_or(mfail);   // every thread takes the same value
    }
    // after an error, B loads still in flight land before the block exits
    if (TMA && b_pending) (void)mbar_wait(smem_u32(&mbar_b), (phase_b - 1) & 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // partial R of this block's taps: warp q (mod 4) reads lanes 32q..32q+31
    // (a = 32q + lane); the two warpgroups take alternate 8-column chunks
    if (ok) {
        const int q = warp & 3, half = warp >> 2;
        const int a = 32 * q + lane;
        const int ncol = (t1 - t0) * cb;
        for (int c0 = 8 * half; c0 < ncol; c0 += 16) {
            float v[8];
            if (!first) tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
            else
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = 0.0f;
            if (a < ca) {
                const int t = t0 + c0 / cb, b = c0 % cb;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    part[(((size_t)blockIdx.x * ca + a) * cb + b + j) * 27 + t] = v[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
}

// Tile geometry of the weight gradient over A's grid (wa x ha lines): the
// tallest tile whose A rows (16 groups of 8 channels, nk positions) and B box
// fit the shared-memory cap; B rows cover the largest tap shift past the
// last K step.
static bool choose_wgrad_geom(int S, int wa, int ha, int cb, WgGeom *out) {
    bool found = false;
    for (int ty = 1; ty <= kTcMaxTY && ty <= ha; ++ty) {
        WgGeom g;
        g.ty = ty;
        int shift_max;
        if (S == 2) {
            g.ly = ty + 1;
            g.pz = 2;
            g.w2 = wa + 1;
            g.rsub = (g.pz * g.ly * g.w2 + 7) & ~7;
            g.rows = 8 * g.rsub;
            shift_max = 7 * g.rsub;
        } else {
            g.ly = ty + 2;
            g.pz = 3;
            g.w2 = wa + 2;
            g.rsub = g.pz * g.ly * g.w2;
            g.rows = g.rsub;
            shift_max = g.ly * g.w2 + g.w2 + 1;
        }
        g.base = g.ly * g.w2 + g.w2 + 1;
        g.nk = (ty * g.w2 + 15) & ~15;
        const int need = g.base + shift_max + g.nk;
        g.rows_pad = ((need > g.rows ? need : g.rows) + 7) & ~7;
        g.smem = (size_t)16 * g.nk * 16 + (size_t)(cb / 8) * g.rows_pad * 16;
        g.taps_per_group = 512 / cb < 27 ? 512 / cb : 27;
        g.n_groups = (27 + g.taps_per_group - 1) / g.taps_per_group;
        g.tmem_cols = pow2_at_least(g.taps_per_group * cb);
        if (g.smem > kTcSmemCap || g.tmem_cols > 512 || g.rows_pad >= 16384 || g.nk >= 16384) continue;
        *out = g;                        // taller tiles stage fewer halo rows per position
        found = true;
    }
    return found;
}

struct WgradPlan {
    int S, ca, cb, a_is_co, nx;
    const float *A, *B;
    TcDims da, db;
    WgGeom g;
    bool tma;                // B staged by tensor-map box loads from a BF16 copy
    size_t part_bytes;       // per-block partials, rounded up to 256 bytes
    size_t b16_bytes;        // the BF16 8-channel-interleaved copy of B (TMA only)
};

static fe_status wgrad_plan(int mode, const float *d_x, int cin, const int *dims_in, const float *d_dy, int cout,
                            const int *dims_out, WgradPlan *p) {
    if (mode != FE_NN_S1 && mode != FE_NN_S2 && mode != FE_NN_T2) return FE_ERR_ARG;
    if (cin < 1 || cout < 1 || !dims_in || !dims_out) return FE_ERR_ARG;
    for (int i = 0; i < 3; ++i) {
        if (dims_in[i] < 1) return FE_ERR_ARG;
        const int want = mode == FE_NN_S1 ? dims_in[i]
                                          : (mode == FE_NN_S2 ? (dims_in[i] - 1) / 2 + 1 : 2 * (dims_in[i] - 1) + 1);
        if (dims_out[i] != want) return FE_ERR_ARG;
    }
    // S1, S2: R[co][ci][t] = sum_z dY[co][z] X[ci][s z + d - 1]; T2: R[ci][co][t] = sum_z X[ci][z] dY[co][2 z + d - 1]
    const bool t2 = mode == FE_NN_T2;
    p->S = mode == FE_NN_S1 ? 1 : 2;
    p->A = t2 ? d_x : d_dy;
    p->B = t2 ? d_dy : d_x;
    p->ca = t2 ? cin : cout;
    p->cb = t2 ? cout : cin;
    p->a_is_co = t2 ? 0 : 1;
    const int *da = t2 ? dims_in : dims_out, *db = t2 ? dims_out : dims_in;
    p->da = TcDims{da[0], da[1], da[2]};
    p->db = TcDims{db[0], db[1], db[2]};
    if (p->ca > 128 || (p->cb != 16 && p->cb != 32 && p->cb != 64)) return FE_ERR_ARG;
    if (!choose_wgrad_geom(p->S, da[2], da[1], p->cb, &p->g)) return FE_ERR_ARG;
    const int ntiles = da[0] * ((da[1] + p->g.ty - 1) / p->g.ty);
    int nx = sm_count() / p->g.n_groups;
    if (nx < 1) nx = 1;
    if (nx > ntiles) nx = ntiles;
    p->nx = nx;
    // B's box by tensor map when each box dimension (elements traversed) fits 256
    const int bx = p->S == 2 ? 2 * p->g.w2 : p->g.w2, by = p->S == 2 ? 2 * p->g.ly : p->g.ly;
    p->tma = bx <= 256 && by <= 256;
    p->part_bytes = ((size_t)nx * p->ca * p->cb * 27 * sizeof(float) + 255) & ~(size_t)255;
    p->b16_bytes = p->tma ? (size_t)(p->cb / 8) * db[0] * db[1] * db[2] * 16 : 0;
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_nn_mma_image_bytes(int cin, int cout, size_t *h_bytes) {
    if (cin < 1 || cout < 1 || !h_bytes) return FE_ERR_ARG;
    *h_bytes = (size_t)((cin + 15) / 16) * 27 * 2 * cout * 16;
    return FE_OK;
}

fe_status fe_nn_pack_weights_mma(const void *d_w16, int cin, int cout, void *d_img, fe_stream_t stream) {
    if (!d_w16 || !d_img || cin < 1 || cout < 1 || !aligned(d_img, 16)) return FE_ERR_ARG;
    const size_t n = (size_t)((cin + 15) / 16) * 27 * 2 * cout * 8;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_pack_mma<<<blocks, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)d_w16, cin, cout,
                                                         (__nv_bfloat16 *)d_img, n);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_conv3d_s1_tc(const float *d_in, int cin, const int *h_dims, const void *d_img,
                             const float *d_bias, float *d_out, int cout, int relu, fe_stream_t stream) {
    if (!d_in || !d_img || !d_out || cin < 1 || !h_dims || h_dims[0] < 1 || h_dims[1] < 1 || h_dims[2] < 1)
        return FE_ERR_ARG;
    return launch_tc<FE_NN_S1, false>(d_in, nullptr, cin, h_dims, d_img, d_bias, d_out, cout, h_dims, relu,
                                      (cudaStream_t)stream);
}

fe_status fe_nn_conv3d_t2_tc(const float *d_in, int cin, const int *h_dims_in, const void *d_img,
                             const float *d_bias, float *d_out, int cout, const int *h_dims_out, int relu,
                             fe_stream_t stream) {
    if (!d_in || !d_img || !d_out || cin < 1 || !h_dims_in || !h_dims_out) return FE_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (h_dims_in[i] < 1 || h_dims_out[i] != 2 * (h_dims_in[i] - 1) + 1) return FE_ERR_ARG;
    return launch_tc<FE_NN_T2, false>(d_in, nullptr, cin, h_dims_in, d_img, d_bias, d_out, cout, h_dims_out, relu,
                                      (cudaStream_t)stream);
}

fe_status fe_nn_conv3d_s2_tc(const float *d_in, int cin, const int *h_dims_in, const void *d_img,
                             const float *d_bias, float *d_out, int cout, const int *h_dims_out, int relu,
                             fe_stream_t stream) {
    if (!d_in || !d_img || !d_out || cin < 1 || !h_dims_in || !h_dims_out) return FE_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (h_dims_in[i] < 1 || h_dims_out[i] != (h_dims_in[i] - 1) / 2 + 1) return FE_ERR_ARG;
    return launch_tc<FE_NN_S2, false>(d_in, nullptr, cin, h_dims_in, d_img, d_bias, d_out, cout, h_dims_out, relu,
                                      (cudaStream_t)stream);
}

fe_status fe_nn_bf16i_bytes(int c, const int *h_dims, size_t *h_bytes) {
    if (c < 1 || !h_dims || !h_bytes || h_dims[0] < 1 || h_dims[1] < 1 || h_dims[2] < 1) return FE_ERR_ARG;
    *h_bytes = (size_t)((c + 7) / 8) * h_dims[0] * h_dims[1] * h_dims[2] * 16;
    return FE_OK;
}

fe_status fe_nn_to_bf16i(const float *d_in, int c, const int *h_dims, void *d_out, fe_stream_t stream) {
    if (!d_in || !d_out || c < 1 || !h_dims || h_dims[0] < 1 || h_dims[1] < 1 || h_dims[2] < 1) return FE_ERR_ARG;
    if (!aligned(d_out, 16)) return FE_ERR_ARG;
    const size_t v = (size_t)h_dims[0] * h_dims[1] * h_dims[2];
    const size_t n = (size_t)((c + 7) / 8) * v;
    const int blocks = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    k_to_bf16i<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_in, c, v, (__nv_bfloat16 *)d_out);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_conv3d_tc_bf16i(int mode, const void *d_in16, int cin, const int *h_dims_in, const void *d_img,
                                const float *d_bias, float *d_out, int cout, const int *h_dims_out, int relu,
                                fe_stream_t stream) {
    if (!d_in16 || !d_img || !d_out || cin < 1 || !h_dims_in || !h_dims_out) return FE_ERR_ARG;
    if (!aligned(d_in16, 16)) return FE_ERR_ARG;
    for (int i = 0; i < 3; ++i) {
        if (h_dims_in[i] < 1) return FE_ERR_ARG;
        const int want = mode == FE_NN_S1 ? h_dims_in[i]
                                          : (mode == FE_NN_S2 ? (h_dims_in[i] - 1) / 2 + 1 : 2 * (h_dims_in[i] - 1) + 1);
        if (h_dims_out[i] != want) return FE_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == FE_NN_S1)
        return launch_tc<FE_NN_S1, true>(nullptr, d_in16, cin, h_dims_in, d_img, d_bias, d_out, cout, h_dims_out, relu, s);
    if (mode == FE_NN_S2)
        return launch_tc<FE_NN_S2, true>(nullptr, d_in16, cin, h_dims_in, d_img, d_bias, d_out, cout, h_dims_out, relu, s);
    if (mode == FE_NN_T2)
        return launch_tc<FE_NN_T2, true>(nullptr, d_in16, cin, h_dims_in, d_img, d_bias, d_out, cout, h_dims_out, relu, s);
    return FE_ERR_ARG;
}

fe_status fe_nn_wgrad_tc_workspace(int mode, int cin, const int *h_dims_in, int cout, const int *h_dims_out,
                                   size_t *h_bytes) {
    if (!h_bytes) return FE_ERR_ARG;
    WgradPlan p;
    const float dummy = 0.0f;
    fe_status st = wgrad_plan(mode, &dummy, cin, h_dims_in, &dummy, cout, h_dims_out, &p);
    if (st != FE_OK) return st;
    *h_bytes = p.part_bytes + p.b16_bytes;
    return FE_OK;
}

fe_status fe_nn_conv3d_weight_grad_tc(int mode, const float *d_x, int cin, const int *h_dims_in,
                                      const float *d_dy, int cout, const int *h_dims_out, float *d_dw,
                                      float *d_work, size_t work_bytes, fe_stream_t stream) {
    if (!d_x || !d_dy || !d_dw || !d_work) return FE_ERR_ARG;
    WgradPlan p;
    fe_status st = wgrad_plan(mode, d_x, cin, h_dims_in, d_dy, cout, h_dims_out, &p);
    if (st != FE_OK) return st;
    if (work_bytes < p.part_bytes + p.b16_bytes) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    // one block per SM: request enough shared memory that no second block
    // (and no second 512-column tensor-memory allocation) shares it
    size_t smem = p.g.smem;
    if (smem < (size_t)120 * 1024) smem = (size_t)120 * 1024;
    const dim3 grid((unsigned)p.nx, (unsigned)p.g.n_groups);
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    if (p.tma) {
        // B as BF16 [cb/8][D][H][W][8] after the partials, then its box tensor map
        void *b16 = reinterpret_cast<unsigned char *>(d_work) + p.part_bytes;
        if (!aligned(b16, 16)) return FE_ERR_ARG;
        const int dims_b[3] = {p.db.d, p.db.h, p.db.w};
        const size_t v = (size_t)p.db.d * p.db.h * p.db.w;
        const size_t n = (size_t)(p.cb / 8) * v;
        const int blocks = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
        k_to_bf16i<<<blocks, 256, 0, s>>>(p.B, p.cb, v, (__nv_bfloat16 *)b16);
        FE_TRY_LAUNCH();
        if (!encode_box_map(&tm, p.S == 2, b16, p.cb, dims_b, p.g.w2, p.g.ly, p.g.pz)) return FE_ERR_CUDA;
    }
    if (p.S == 1 && p.tma) {
        FE_TRY_CUDA(cudaFuncSetAttribute(k_wgrad_tc<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_wgrad_tc<1, true><<<grid, kTcThreads, smem, s>>>(p.A, p.ca, p.da, p.B, p.cb, p.db, d_work, p.g, tm);
    } else if (p.S == 1) {
        FE_TRY_CUDA(cudaFuncSetAttribute(k_wgrad_tc<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_wgrad_tc<1, false><<<grid, kTcThreads, smem, s>>>(p.A, p.ca, p.da, p.B, p.cb, p.db, d_work, p.g, tm);
    } else if (p.tma) {
        FE_TRY_CUDA(cudaFuncSetAttribute(k_wgrad_tc<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_wgrad_tc<2, true><<<grid, kTcThreads, smem, s>>>(p.A, p.ca, p.da, p.B, p.cb, p.db, d_work, p.g, tm);
    } else {
        FE_TRY_CUDA(cudaFuncSetAttribute(k_wgrad_tc<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_wgrad_tc<2, false><<<grid, kTcThreads, smem, s>>>(p.A, p.ca, p.da, p.B, p.cb, p.db, d_work, p.g, tm);
    }
    FE_TRY_LAUNCH();
    return launch_corr_reduce(d_work, p.nx, p.ca, p.cb, p.a_is_co, d_dw, s);
}

fe_status fe_nn_tc_check(int *h_flag) {
    if (!h_flag) return FE_ERR_ARG;
    int zero = 0;
    FE_TRY_CUDA(cudaMemcpyFromSymbol(h_flag, g_tc_err, sizeof(int)));
    FE_TRY_CUDA(cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(int)));
    return FE_OK;
}

}  // extern "C"
