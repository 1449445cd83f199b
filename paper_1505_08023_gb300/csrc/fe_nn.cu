// fe_nn.cu -- kernels of the learned warm start (a 3-D convolutional
// encoder-decoder that predicts the CG start vector from the Dirichlet face
// data; not in the paper; the FP64 solve from that vector decides convergence).
//
// Activations are FP32 [C][D][H][W] volumes (W fastest), one sample at a time.
// Every 3x3x3 convolution is written in one "gather" form
//     out[co][u] = bias[co] + sum_ci sum_t W[ci][t][co] * in[ci][src(u, t)]
// with tap t = 9 dz + 3 dy + dx and, per axis,
//     FE_NN_S1  src = u + d - 1            (stride 1, same grid)
//     FE_NN_S2  src = 2u + d - 1           (stride 2, fine -> coarse)
//     FE_NN_T2  src = (u + 1 - d) / 2      (transposed stride 2, coarse -> fine;
//                                           only taps where this is an integer)
// and zero outside the input grid.  T2 with weights W'[co][t][ci] = W[ci][t][co]
// is the adjoint of S2 with W, and S1 with taps flipped (t -> 26 - t) and
// channels swapped is the adjoint of S1, so the data gradient of every layer
// is one more forward launch with a transposed weight copy.  Weight gradients
// are correlations R[a][b][t] = sum_z A[a][z] B[b][s z + d - 1], split over
// voxel tiles and summed in a fixed order.  Weights are used in BF16 (rounded
// from FP32 master weights), all accumulation is FP32.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "fe_common.cuh"

namespace fe {

constexpr int kNnThreads = 256;
constexpr int kCoTile = 16;      // output channels per block (forward)
constexpr int kCiChunk = 4;      // input channels staged per round (forward)

__host__ __device__ constexpr int tile_z() { return 4; }
__host__ __device__ constexpr int tile_y() { return 8; }
__host__ __device__ constexpr int tile_x() { return 8; }

// input extent and origin of a stride-2 output tile, per axis
__host__ __device__ constexpr int s2_extent(int t) { return 2 * t + 1; }
__device__ __forceinline__ int s2_origin(int u0) { return 2 * u0 - 1; }

struct Dims {
    int d, h, w;
};

// Stride-2 forward on CUDA cores (the FP32 reference path): thread = one
// output voxel x 16 output channels, input halo tile and BF16 weights staged
// in shared memory per 4-channel chunk.
__global__ void __launch_bounds__(kNnThreads)
k_conv_fwd_s2(const float *__restrict__ in, int cin, Dims di, const __nv_bfloat16 *__restrict__ wt,
              const float *__restrict__ bias, float *__restrict__ out, int cout, Dims dout, int relu) {
    constexpr int TZ = tile_z(), TY = tile_y(), TX = tile_x();
    constexpr int EZ = s2_extent(TZ), EY = s2_extent(TY), EX = s2_extent(TX);
    constexpr int EV = EZ * EY * EX;
    __shared__ float s_in[kCiChunk][EV];
    __shared__ __align__(16) float s_w[kCiChunk][27][kCoTile];

    const int tiles_x = (dout.w + TX - 1) / TX, tiles_y = (dout.h + TY - 1) / TY;
    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int co0 = blockIdx.y * kCoTile;
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    const int ux = bx * TX + tx, uy = by * TY + ty, uz = bz * TZ + tz;
    const int oz = s2_origin(bz * TZ), oy = s2_origin(by * TY), ox = s2_origin(bx * TX);

    float acc[kCoTile];
#pragma unroll
    for (int c = 0; c < kCoTile; ++c) acc[c] = 0.0f;

    for (int ci0 = 0; ci0 < cin; ci0 += kCiChunk) {
        // stage the input halo tile (zero outside the grid) and the weights
        for (int i = threadIdx.x; i < kCiChunk * EV; i += kNnThreads) {
            const int c = i / EV, e = i % EV;
            const int ex = e % EX, ey = (e / EX) % EY, ez = e / (EX * EY);
            const int gx = ox + ex, gy = oy + ey, gz = oz + ez;
            float v = 0.0f;
            if (ci0 + c < cin && gx >= 0 && gx < di.w && gy >= 0 && gy < di.h && gz >= 0 && gz < di.d)
                v = in[((size_t)(ci0 + c) * di.d + gz) * di.h * di.w + (size_t)gy * di.w + gx];
            s_in[c][e] = v;
        }
        for (int i = threadIdx.x; i < kCiChunk * 27 * kCoTile; i += kNnThreads) {
            const int co = i % kCoTile, tap = (i / kCoTile) % 27, c = i / (kCoTile * 27);
            float v = 0.0f;
            if (ci0 + c < cin && co0 + co < cout)
                v = __bfloat162float(wt[((size_t)(ci0 + c) * 27 + tap) * cout + co0 + co]);
            s_w[c][tap][co] = v;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kCiChunk; ++c) {
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                const int lz = 2 * tz + dz, ly = 2 * ty + dy, lx = 2 * tx + dx;
                const float v = s_in[c][(lz * EY + ly) * EX + lx];
                const float4 *w4 = reinterpret_cast<const float4 *>(&s_w[c][tap][0]);
#pragma unroll
                for (int q = 0; q < kCoTile / 4; ++q) {
                    const float4 w = w4[q];
                    acc[4 * q + 0] = fmaf(w.x, v, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(w.y, v, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(w.z, v, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(w.w, v, acc[4 * q + 3]);
                }
            }
        }
        __syncthreads();
    }
    if (ux < dout.w && uy < dout.h && uz < dout.d) {
        const size_t vox = ((size_t)uz * dout.h + uy) * dout.w + ux;
        const size_t plane = (size_t)dout.d * dout.h * dout.w;
#pragma unroll
        for (int c = 0; c < kCoTile; ++c) {
            if (co0 + c >= cout) break;
            float y = acc[c] + (bias ? bias[co0 + c] : 0.0f);
            if (relu) y = y > 0.0f ? y : 0.0f;
            out[(size_t)(co0 + c) * plane + vox] = y;
        }
    }
}

// Stride-1 forward, register-blocked: each thread computes 4 consecutive
// voxels along x for 16 output channels.  For a (ci, dz, dy) the 6 input
// values x-1 .. x+4 serve all three dx taps of the 4 voxels, so one input
// load feeds 8 FMAs and one broadcast float4 weight load feeds 16.
constexpr int kV = 4;
constexpr int kS1TZ = 4, kS1TY = 8, kS1TX = 8 * kV;   // 256 threads x 4 voxels

__global__ void __launch_bounds__(kNnThreads)
k_conv_fwd_s1v(const float *__restrict__ in, int cin, Dims di, const __nv_bfloat16 *__restrict__ wt,
               const float *__restrict__ bias, float *__restrict__ out, int cout, Dims dout, int relu) {
    constexpr int EZ = kS1TZ + 2, EY = kS1TY + 2, EX = kS1TX + 2;
    constexpr int EV = EZ * EY * EX;
    __shared__ float s_in[kCiChunk][EV];
    __shared__ __align__(16) float s_w[kCiChunk][27][kCoTile];
    const int tiles_x = (dout.w + kS1TX - 1) / kS1TX, tiles_y = (dout.h + kS1TY - 1) / kS1TY;
    int t = blockIdx.x;
    const int bx = t % tiles_x;
    t /= tiles_x;
    const int by = t % tiles_y;
    const int bz = t / tiles_y;
    const int co0 = blockIdx.y * kCoTile;
    const int tx = threadIdx.x % 8, ty = (threadIdx.x / 8) % kS1TY, tz = threadIdx.x / (8 * kS1TY);
    const int ux0 = bx * kS1TX + kV * tx, uy = by * kS1TY + ty, uz = bz * kS1TZ + tz;
    const int oz = bz * kS1TZ - 1, oy = by * kS1TY - 1, ox = bx * kS1TX - 1;
    float acc[kV][kCoTile];
#pragma unroll
    for (int v = 0; v < kV; ++v)
#pragma unroll
        for (int c = 0; c < kCoTile; ++c) acc[v][c] = 0.0f;
    for (int ci0 = 0; ci0 < cin; ci0 += kCiChunk) {
        for (int i = threadIdx.x; i < kCiChunk * EV; i += kNnThreads) {
            const int c = i / EV, e = i % EV;
            const int ex = e % EX, ey = (e / EX) % EY, ez = e / (EX * EY);
            const int gx = ox + ex, gy = oy + ey, gz = oz + ez;
            float v = 0.0f;
            if (ci0 + c < cin && gx >= 0 && gx < di.w && gy >= 0 && gy < di.h && gz >= 0 && gz < di.d)
                v = in[((size_t)(ci0 + c) * di.d + gz) * di.h * di.w + (size_t)gy * di.w + gx];
            s_in[c][e] = v;
        }
        for (int i = threadIdx.x; i < kCiChunk * 27 * kCoTile; i += kNnThreads) {
            const int co = i % kCoTile, tap = (i / kCoTile) % 27, c = i / (kCoTile * 27);
            float v = 0.0f;
            if (ci0 + c < cin && co0 + co < cout)
                v = __bfloat162float(wt[((size_t)(ci0 + c) * 27 + tap) * cout + co0 + co]);
            s_w[c][tap][co] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < kCiChunk; ++c) {
#pragma unroll
            for (int dzy = 0; dzy < 9; ++dzy) {
                const int dz = dzy / 3, dy = dzy % 3;
                const float *row = &s_in[c][((tz + dz) * EY + ty + dy) * EX + kV * tx];
                float xv[kV + 2];
#pragma unroll
                for (int k = 0; k < kV + 2; ++k) xv[k] = row[k];
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float4 *w4 = reinterpret_cast<const float4 *>(&s_w[c][dzy * 3 + dx][0]);
#pragma unroll
                    for (int q = 0; q < kCoTile / 4; ++q) {
                        const float4 w = w4[q];
#pragma unroll
                        for (int v = 0; v < kV; ++v) {
                            const float xin = xv[v + dx];
                            acc[v][4 * q + 0] = fmaf(w.x, xin, acc[v][4 * q + 0]);
                            acc[v][4 * q + 1] = fmaf(w.y, xin, acc[v][4 * q + 1]);
                            acc[v][4 * q + 2] = fmaf(w.z, xin, acc[v][4 * q + 2]);
                            acc[v][4 * q + 3] = fmaf(w.w, xin, acc[v][4 * q + 3]);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (uy < dout.h && uz < dout.d) {
        const size_t plane = (size_t)dout.d * dout.h * dout.w;
        const size_t vrow = ((size_t)uz * dout.h + uy) * dout.w;
#pragma unroll
        for (int c = 0; c < kCoTile; ++c) {
            if (co0 + c >= cout) break;
            const float bc = bias ? bias[co0 + c] : 0.0f;
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                if (ux0 + v >= dout.w) break;
                float y = acc[v][c] + bc;
                if (relu) y = y > 0.0f ? y : 0.0f;
                out[(size_t)(co0 + c) * plane + vrow + ux0 + v] = y;
            }
        }
    }
}

// Transposed stride-2 forward by output parity class.  Output u = 2v + p
// (p = 0 or 1 per axis) receives, per axis, tap d = 1 from input v when p = 0,
// and taps d = 0 (input v + 1) and d = 2 (input v) when p = 1.  A block works
// on one class (blockIdx.z), so every thread runs the same 1..8 taps with no
// parity test; each thread computes 4 consecutive v along x x 16 channels.
constexpr int kT2TZ = 4, kT2TY = 8, kT2TX = 8 * kV;

__global__ void __launch_bounds__(kNnThreads)
k_conv_fwd_t2p(const float *__restrict__ in, int cin, Dims di, const __nv_bfloat16 *__restrict__ wt,
               const float *__restrict__ bias, float *__restrict__ out, int cout, Dims dout, int relu) {
    constexpr int EZ = kT2TZ + 1, EY = kT2TY + 1, EX = kT2TX + 1;
    constexpr int EV = EZ * EY * EX;
    __shared__ float s_in[kCiChunk][EV];
    __shared__ __align__(16) float s_w[kCiChunk][27][kCoTile];
    const int pz = (blockIdx.z >> 2) & 1, py = (blockIdx.z >> 1) & 1, px = blockIdx.z & 1;
    // class sub-grid sizes: v with 2v + p < D
    const int cz = (dout.d - pz + 1) / 2, cy = (dout.h - py + 1) / 2, cx = (dout.w - px + 1) / 2;
    const int tiles_x = (cx + kT2TX - 1) / kT2TX, tiles_y = (cy + kT2TY - 1) / kT2TY;
    // the grid is sized for the largest class (p = 0); smaller classes skip extra tiles
    const int full_x = ((dout.w + 1) / 2 + kT2TX - 1) / kT2TX, full_y = ((dout.h + 1) / 2 + kT2TY - 1) / kT2TY;
    int t = blockIdx.x;
    const int bx = t % full_x;
    t /= full_x;
    const int by = t % full_y;
    const int bz = t / full_y;
    if (bx >= tiles_x || by >= tiles_y || bz * kT2TZ >= cz) return;
    const int co0 = blockIdx.y * kCoTile;
    const int tx = threadIdx.x % 8, ty = (threadIdx.x / 8) % kT2TY, tz = threadIdx.x / (8 * kT2TY);
    const int v0z = bz * kT2TZ, v0y = by * kT2TY, v0x = bx * kT2TX;
    const int nz = pz ? 2 : 1, ny = py ? 2 : 1, nxt = px ? 2 : 1;
    float acc[kV][kCoTile];
#pragma unroll
    for (int v = 0; v < kV; ++v)
#pragma unroll
        for (int c = 0; c < kCoTile; ++c) acc[v][c] = 0.0f;
    for (int ci0 = 0; ci0 < cin; ci0 += kCiChunk) {
        for (int i = threadIdx.x; i < kCiChunk * EV; i += kNnThreads) {
            const int c = i / EV, e = i % EV;
            const int ex = e % EX, ey = (e / EX) % EY, ez = e / (EX * EY);
            const int gx = v0x + ex, gy = v0y + ey, gz = v0z + ez;
            float v = 0.0f;
            if (ci0 + c < cin && gx < di.w && gy < di.h && gz < di.d)
                v = in[((size_t)(ci0 + c) * di.d + gz) * di.h * di.w + (size_t)gy * di.w + gx];
            s_in[c][e] = v;
        }
        for (int i = threadIdx.x; i < kCiChunk * 27 * kCoTile; i += kNnThreads) {
            const int co = i % kCoTile, tap = (i / kCoTile) % 27, c = i / (kCoTile * 27);
            float v = 0.0f;
            if (ci0 + c < cin && co0 + co < cout)
                v = __bfloat162float(wt[((size_t)(ci0 + c) * 27 + tap) * cout + co0 + co]);
            s_w[c][tap][co] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < kCiChunk; ++c) {
            for (int iz = 0; iz < nz; ++iz) {
                const int dz = pz ? 2 * iz : 1, oz = pz ? 1 - iz : 0;
                for (int iy = 0; iy < ny; ++iy) {
                    const int dy = py ? 2 * iy : 1, oy = py ? 1 - iy : 0;
                    const float *row = &s_in[c][((tz + oz) * EY + ty + oy) * EX + kV * tx];
                    float xv[kV + 1];
#pragma unroll
                    for (int k = 0; k < kV + 1; ++k) xv[k] = row[k];
                    for (int ix = 0; ix < nxt; ++ix) {
                        const int dx = px ? 2 * ix : 1, ox = px ? 1 - ix : 0;
                        const float4 *w4 = reinterpret_cast<const float4 *>(&s_w[c][dz * 9 + dy * 3 + dx][0]);
#pragma unroll
                        for (int q = 0; q < kCoTile / 4; ++q) {
                            const float4 w = w4[q];
#pragma unroll
                            for (int v = 0; v < kV; ++v) {
                                const float xin = ox ? xv[v + 1] : xv[v];
                                acc[v][4 * q + 0] = fmaf(w.x, xin, acc[v][4 * q + 0]);
                                acc[v][4 * q + 1] = fmaf(w.y, xin, acc[v][4 * q + 1]);
                                acc[v][4 * q + 2] = fmaf(w.z, xin, acc[v][4 * q + 2]);
                                acc[v][4 * q + 3] = fmaf(w.w, xin, acc[v][4 * q + 3]);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    const int vz = v0z + tz, vy = v0y + ty;
    if (vz < cz && vy < cy) {
        const int uz = 2 * vz + pz, uy = 2 * vy + py;
        const size_t plane = (size_t)dout.d * dout.h * dout.w;
        const size_t vrow = ((size_t)uz * dout.h + uy) * dout.w;
#pragma unroll
        for (int c = 0; c < kCoTile; ++c) {
            if (co0 + c >= cout) break;
            const float bc = bias ? bias[co0 + c] : 0.0f;
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const int vx = v0x + kV * tx + v;
                if (vx >= cx) break;
                float y = acc[v][c] + bc;
                if (relu) y = y > 0.0f ? y : 0.0f;
                out[(size_t)(co0 + c) * plane + vrow + 2 * vx + px] = y;
            }
        }
    }
}

// Weight gradient, register-blocked: R[a][b][t] = sum_z A[a][z] B[b][S z + d_t - 1].
// Each thread accumulates 4 consecutive a x one b x 27 taps; a block has
// ag a-groups x bt b's x zs voxel sub-splits (ag bt zs = 256), fitted to the
// channel counts so that few threads idle when a layer has few channels.
// The sub-splits are summed in the block; each block (or each warp, when a
// block has more than 32 sub-splits) writes one partial; k_corr_reduce sums them.
struct CorrShape {
    int ag, bt, zs;
};
constexpr int kCorrMaxB = 16;

template <int S>
__global__ void __launch_bounds__(kNnThreads, 2)   // 2 blocks/SM: one stages while the other computes
k_corr4(const float *__restrict__ A, int ca, Dims da, const float *__restrict__ B, int cb, Dims dbg,
        float *__restrict__ part, int n_split, CorrShape cs) {
    constexpr int TZ = 2, TY = (S == 1) ? 8 : 2, TX = 8;
    constexpr int EZ = S * TZ + 2 - (S - 1), EY = S * TY + 2 - (S - 1), EX = S * TX + 2 - (S - 1);
    constexpr int EV = EZ * EY * EX, NV = TZ * TY * TX;
    constexpr int MAXA = 16, MAXB = kCorrMaxB;  // 34 KB (S = 1) / 29 KB (S = 2) of static shared memory
    __shared__ __align__(16) float s_a[NV][MAXA];   // [voxel][a]: one float4 per a-group
    __shared__ float s_b[MAXB][EV];
    const int at = 4 * cs.ag;
    const int tid = threadIdx.x;
    const int zsub = tid % cs.zs, rest = tid / cs.zs;
    const int ib = rest % cs.bt, ig = rest / cs.bt;
    const int n_bt = (cb + cs.bt - 1) / cs.bt;
    const int a0 = (blockIdx.y / n_bt) * at, b0 = (blockIdx.y % n_bt) * cs.bt;
    const int tiles_x = (da.w + TX - 1) / TX, tiles_y = (da.h + TY - 1) / TY, tiles_z = (da.d + TZ - 1) / TZ;
    const int n_tiles = tiles_x * tiles_y * tiles_z;
    float acc[4][27];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int t = 0; t < 27; ++t) acc[k][t] = 0.0f;
    for (int tile = blockIdx.x; tile < n_tiles; tile += n_split) {
        const int bx = tile % tiles_x, by = (tile / tiles_x) % tiles_y, bz = tile / (tiles_x * tiles_y);
        const int z0 = bz * TZ, y0 = by * TY, x0 = bx * TX;
        for (int i = tid; i < NV * MAXA; i += kNnThreads) {
            const int e = i / MAXA, c = i % MAXA;
            const int ex = e % TX, ey = (e / TX) % TY, ez = e / (TX * TY);
            const int gx = x0 + ex, gy = y0 + ey, gz = z0 + ez;
            float v = 0.0f;
            if (c < at && a0 + c < ca && gx < da.w && gy < da.h && gz < da.d)
                v = A[((size_t)(a0 + c) * da.d + gz) * da.h * da.w + (size_t)gy * da.w + gx];
            s_a[e][c] = v;
        }
        const int oz = S * z0 - 1, oy = S * y0 - 1, ox = S * x0 - 1;
        for (int i = tid; i < cs.bt * EV; i += kNnThreads) {
            const int c = i / EV, e = i % EV;
            const int ex = e % EX, ey = (e / EX) % EY, ez = e / (EX * EY);
            const int gx = ox + ex, gy = oy + ey, gz = oz + ez;
            float v = 0.0f;
            if (b0 + c < cb && gx >= 0 && gx < dbg.w && gy >= 0 && gy < dbg.h && gz >= 0 && gz < dbg.d)
                v = B[((size_t)(b0 + c) * dbg.d + gz) * dbg.h * dbg.w + (size_t)gy * dbg.w + gx];
            s_b[c][e] = v;
        }
        __syncthreads();
        for (int e = zsub; e < NV; e += cs.zs) {
            const float4 av = *reinterpret_cast<const float4 *>(&s_a[e][4 * ig]);
            const int ex = e % TX, ey = (e / TX) % TY, ez = e / (TX * TY);
            const float *bb = &s_b[ib][((S * ez) * EY + S * ey) * EX + S * ex];
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                const float bv = bb[(dz * EY + dy) * EX + dx];
                acc[0][t] = fmaf(av.x, bv, acc[0][t]);
                acc[1][t] = fmaf(av.y, bv, acc[1][t]);
                acc[2][t] = fmaf(av.z, bv, acc[2][t]);
                acc[3][t] = fmaf(av.w, bv, acc[3][t]);
            }
        }
        __syncthreads();
    }
    // Sum the sub-splits: they are the low log2(zs) bits of the thread index,
    // so within a warp a fixed xor butterfly combines them; when zs > 32 each
    // warp's sum is its own partial (zs / 32 per block).
    for (int off = 1; off < cs.zs && off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int t = 0; t < 27; ++t) acc[k][t] += __shfl_xor_sync(0xffffffffu, acc[k][t], off);
    }
    if ((zsub & 31) != 0) return;
    const int per_block = cs.zs > 32 ? cs.zs / 32 : 1;
    const int split = blockIdx.x * per_block + (zsub >> 5);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = a0 + 4 * ig + k, b = b0 + ib;
        if (a < ca && b < cb) {
            float *p = part + (((size_t)split * ca + a) * cb + b) * 27;
#pragma unroll
            for (int t = 0; t < 27; ++t) p[t] = acc[k][t];
        }
    }
}

// ag a-groups of 4 channels (1, 2 or 4), bt b-channels (power of 2, at most
// kCorrMaxB so the B halo tile fits static shared memory), zs voxel sub-splits
// filling 256 threads (a power of 2, so the sub-splits are the low thread bits).
static CorrShape corr_shape(int stride, int ca, int cb) {
    (void)stride;
    CorrShape cs;
    cs.ag = ca > 8 ? 4 : (ca > 4 ? 2 : 1);
    int bt = 1;
    while (bt < cb && bt < kCorrMaxB && cs.ag * bt * 2 <= kNnThreads) bt *= 2;
    cs.bt = bt;
    cs.zs = kNnThreads / (cs.ag * cs.bt);
    return cs;
}

// R = sum over splits (fixed order); scattered into dW[ci][t][co]:
// a_is_co = 1: R[a=co][b=ci][t]; a_is_co = 0: R[a=ci][b=co][t].
// A block covers 32 consecutive outputs (one per lane); warp w sums the
// partials of its contiguous share in order, then warp 0 adds the eight warp
// sums in warp order.
__global__ void __launch_bounds__(kNnThreads)
k_corr_reduce(const float *__restrict__ part, int n_split, int ca, int cb, int a_is_co, float *__restrict__ dw) {
    __shared__ float red[kNnThreads / 32][32];
    const int n = ca * cb * 27;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int per = (n_split + kNnThreads / 32 - 1) / (kNnThreads / 32);
    const int k0 = warp * per, k1 = min(n_split, k0 + per);
    float s = 0.0f;
    if (i < n)
        for (int k = k0; k < k1; ++k) s += part[(size_t)k * n + i];
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && i < n) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < kNnThreads / 32; ++w) tot += red[w][lane];
        const int t = i % 27, b = (i / 27) % cb, a = i / (27 * cb);
        const int ci = a_is_co ? b : a, co = a_is_co ? a : b;
        const int cout = a_is_co ? ca : cb;
        dw[((size_t)ci * 27 + t) * cout + co] = tot;
    }
}

// Bias gradient db[c] = sum over the volume of dy[c].  One cluster of 8
// blocks per channel: block r sums the r-th eighth of the volume (four
// interleaved accumulators per thread, then warps, then warps in order), and
// block 0 adds the eight block sums in rank order through distributed shared
// memory, so the result is fixed for a given volume size.
constexpr int kSumCluster = 8, kSumThreads = 1024;

__global__ void __cluster_dims__(kSumCluster, 1, 1) __launch_bounds__(kSumThreads)
k_channel_sum(const float *__restrict__ dy, size_t plane, float *__restrict__ db) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ float red[kSumThreads / 32];
    __shared__ float block_total;
    const unsigned rank = cluster.block_rank();
    const size_t c = blockIdx.x / kSumCluster;
    const size_t chunk = (plane + kSumCluster - 1) / kSumCluster;
    const size_t lo = rank * chunk, hi = min(plane, lo + chunk);
    const float *p = dy + c * plane;
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    size_t i = lo + threadIdx.x;
    for (; i + 3 * kSumThreads < hi; i += 4 * kSumThreads) {
        s0 += p[i];
        s1 += p[i + kSumThreads];
        s2 += p[i + 2 * kSumThreads];
        s3 += p[i + 3 * kSumThreads];
    }
    for (; i < hi; i += kSumThreads) s0 += p[i];
    float s = warp_sum((s0 + s1) + (s2 + s3));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kSumThreads / 32; ++w) t += red[w];
        block_total = t;
    }
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        float t = 0.0f;
        for (int r = 0; r < kSumCluster; ++r) t += *cluster.map_shared_rank(&block_total, r);
        db[c] = t;
    }
    cluster.sync();   // peers keep their shared memory until block 0 has read it
}

// Weight copies in BF16: forward (same layout) or transposed for the data
// gradient: dst[co][t'][ci] = src[ci][flip ? 26 - t' : t'][co].
__global__ void k_pack_weights(const float *__restrict__ src, int cin, int cout, int transpose,
                               int flip, __nv_bfloat16 *__restrict__ dst) {
    const int n = cin * 27 * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!transpose) {
            dst[i] = __float2bfloat16(src[i]);
        } else {
            const int ci = i % cin, tp = (i / cin) % 27, co = i / (cin * 27);
            const int t = flip ? 26 - tp : tp;
            dst[i] = __float2bfloat16(src[((size_t)ci * 27 + t) * cout + co]);
        }
    }
}

__global__ void k_relu_bwd(const float *__restrict__ y, float *__restrict__ dy, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(y[i] > 0.0f)) dy[i] = 0.0f;
}

__global__ void k_axpy(float a, const float *__restrict__ x, float *__restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]);
}

// 1x1x1 head: out[u] = b + sum_c w[c] h[c][u] (w in BF16)
__global__ void k_head_fwd(const float *__restrict__ h, int c, size_t plane,
                           const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b,
                           float *__restrict__ out) {
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < plane; u += (size_t)gridDim.x * blockDim.x) {
        float s = b[0];
        for (int k = 0; k < c; ++k) s = fmaf(__bfloat162float(w[k]), h[(size_t)k * plane + u], s);
        out[u] = s;
    }
}

// head data gradient dh[c][u] = w[c] dout[u]
__global__ void k_head_bwd_data(const float *__restrict__ dout, int c, size_t plane,
                                const __nv_bfloat16 *__restrict__ w, float *__restrict__ dh) {
    const size_t n = (size_t)c * plane;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dh[i] = __bfloat162float(w[i / plane]) * dout[i % plane];
}

// per-block partial sums of h[c][u] * dout[u] (grid.y = c), fixed order
__global__ void k_head_bwd_weight(const float *__restrict__ h, const float *__restrict__ dout,
                                  size_t plane, float *__restrict__ part) {
    __shared__ float red[kNnThreads / 32];
    const int c = blockIdx.y;
    float s = 0.0f;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < plane; u += (size_t)gridDim.x * blockDim.x)
        s = fmaf(h[(size_t)c * plane + u], dout[u], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kNnThreads / 32; ++w) t += red[w];
        part[(size_t)c * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void k_rows_sum(const float *__restrict__ part, int rows, int cols, float *__restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float s = 0.0f;
    for (int k = 0; k < cols; ++k) s += part[(size_t)r * cols + k];
    out[r] = s;
}

// Loss on interior nodes: mean (pred - target)^2; gradient written to dpred
// (zero on boundary nodes); per-block partials of the squared error.
__global__ void k_mse(const float *__restrict__ pred, const float *__restrict__ target,
                      const uint8_t *__restrict__ bc_flag, size_t n, float scale,
                      float *__restrict__ dpred, float *__restrict__ part) {
    __shared__ float red[kNnThreads / 32];
    float s = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float g = 0.0f;
        if (!bc_flag[i]) {
            const float d = pred[i] - target[i];
            s = fmaf(d, d, s);
            g = 2.0f * scale * d;
        }
        dpred[i] = g;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kNnThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Adam on FP32 master weights (bias-corrected step sizes passed in).
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, size_t n, float lr_t, float b1, float b2, float eps) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr_t * mi / (sqrtf(vi) + eps);
    }
}

// Network input from the mesh: channel 0 = boundary value (0 inside),
// channel 1 = boundary flag.
__global__ void k_ws_input(const uint8_t *__restrict__ bc_flag, const double *__restrict__ bc_val,
                           size_t n, float *__restrict__ x) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const bool b = bc_flag[i] != 0;
        x[i] = b ? (float)bc_val[i] : 0.0f;
        x[n + i] = b ? 1.0f : 0.0f;
    }
}

// Start vector: prescribed value on boundary nodes, prediction inside.
__global__ void k_ws_output(const float *__restrict__ pred, const uint8_t *__restrict__ bc_flag,
                            const double *__restrict__ bc_val, size_t n, double *__restrict__ x0) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x0[i] = bc_flag[i] ? bc_val[i] : (double)pred[i];
}

static int grid1(size_t n) {
    size_t b = (n + kNnThreads - 1) / kNnThreads;
    size_t cap = (size_t)(sm_count() > 0 ? sm_count() : 132) * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

static Dims dims_of(const int *d) { return Dims{d[0], d[1], d[2]}; }

static bool dims_ok(const int *d) { return d && d[0] > 0 && d[1] > 0 && d[2] > 0; }

static bool mode_dims_ok(int mode, const int *din, const int *dout) {
    for (int k = 0; k < 3; ++k) {
        if (mode == FE_NN_S1 && dout[k] != din[k]) return false;
        if (mode == FE_NN_S2 && dout[k] != (din[k] - 1) / 2 + 1) return false;
        if (mode == FE_NN_T2 && dout[k] != 2 * (din[k] - 1) + 1) return false;
    }
    return true;
}

}  // namespace fe

namespace fe {

// dW[ci][t][co] from per-split partials part[split][a][b][t] (fixed order),
// for the tensor-core weight gradient (fe_nn_tc.cu).
fe_status launch_corr_reduce(const float *part, int n_split, int ca, int cb, int a_is_co, float *dw,
                             cudaStream_t s) {
    k_corr_reduce<<<(ca * cb * 27 + 31) / 32, kNnThreads, 0, s>>>(part, n_split, ca, cb, a_is_co, dw);
    FE_TRY_LAUNCH();
    return FE_OK;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_nn_conv3d(int mode, const float *d_in, int cin, const int *dims_in, const void *d_wv,
                       const float *d_bias, float *d_out, int cout, const int *dims_out, int relu,
                       fe_stream_t stream) {
    const __nv_bfloat16 *d_w = (const __nv_bfloat16 *)d_wv;
    if (!d_in || !d_w || !d_out || cin < 1 || cout < 1 || !dims_ok(dims_in) || !dims_ok(dims_out))
        return FE_ERR_ARG;
    if (mode != FE_NN_S1 && mode != FE_NN_S2 && mode != FE_NN_T2) return FE_ERR_ARG;
    if (!mode_dims_ok(mode, dims_in, dims_out)) return FE_ERR_ARG;
    const Dims di = dims_of(dims_in), dout = dims_of(dims_out);
    const int tiles = ((dout.w + tile_x() - 1) / tile_x()) * ((dout.h + tile_y() - 1) / tile_y()) *
                      ((dout.d + tile_z() - 1) / tile_z());
    dim3 grid(tiles, (cout + kCoTile - 1) / kCoTile);
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == FE_NN_S1) {
        const int tv = ((dout.w + kS1TX - 1) / kS1TX) * ((dout.h + kS1TY - 1) / kS1TY) *
                       ((dout.d + kS1TZ - 1) / kS1TZ);
        k_conv_fwd_s1v<<<dim3(tv, (cout + kCoTile - 1) / kCoTile), kNnThreads, 0, s>>>(
            d_in, cin, di, d_w, d_bias, d_out, cout, dout, relu);
    } else if (mode == FE_NN_S2) {
        k_conv_fwd_s2<<<grid, kNnThreads, 0, s>>>(d_in, cin, di, d_w, d_bias, d_out, cout, dout, relu);
    } else {
        const int cz = (dout.d + 1) / 2, cy = (dout.h + 1) / 2, cx = (dout.w + 1) / 2;  // largest class
        const int tv = ((cx + kT2TX - 1) / kT2TX) * ((cy + kT2TY - 1) / kT2TY) * ((cz + kT2TZ - 1) / kT2TZ);
        k_conv_fwd_t2p<<<dim3(tv, (cout + kCoTile - 1) / kCoTile, 8), kNnThreads, 0, s>>>(
            d_in, cin, di, d_w, d_bias, d_out, cout, dout, relu);
    }
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_corr_workspace(int stride, int ca, const int *dims_a, int cb, size_t *h_bytes,
                               int *h_splits) {
    if ((stride != 1 && stride != 2) || ca < 1 || cb < 1 || !dims_ok(dims_a) || !h_bytes) return FE_ERR_ARG;
    const int TZ = 2, TY = stride == 1 ? 8 : 2, TX = 8;
    const long long tiles = (long long)((dims_a[2] + TX - 1) / TX) * ((dims_a[1] + TY - 1) / TY) *
                            ((dims_a[0] + TZ - 1) / TZ);
    const CorrShape cs = corr_shape(stride, ca, cb);
    const long long blocks_yz = (long long)((ca + 4 * cs.ag - 1) / (4 * cs.ag)) * ((cb + cs.bt - 1) / cs.bt);
    long long split = (long long)(sm_count() > 0 ? sm_count() : 132) * 4 / blocks_yz;
    if (split < 1) split = 1;
    if (split > tiles) split = tiles;
    const int per_block = cs.zs > 32 ? cs.zs / 32 : 1;
    *h_bytes = (size_t)split * per_block * ca * cb * 27 * sizeof(float);
    if (h_splits) *h_splits = (int)(split * per_block);
    return FE_OK;
}

fe_status fe_nn_conv3d_weight_grad(int mode, const float *d_x, int cin, const int *dims_in,
                                   const float *d_dy, int cout, const int *dims_out, float *d_dw,
                                   float *d_work, size_t work_bytes, fe_stream_t stream) {
    if (!d_x || !d_dy || !d_dw || !d_work || cin < 1 || cout < 1 || !dims_ok(dims_in) || !dims_ok(dims_out))
        return FE_ERR_ARG;
    if (mode != FE_NN_S1 && mode != FE_NN_S2 && mode != FE_NN_T2) return FE_ERR_ARG;
    if (!mode_dims_ok(mode, dims_in, dims_out)) return FE_ERR_ARG;
    // S1, S2: R[co][ci][t] = sum_z dY[co][z] X[ci][s z + d - 1]  (A = dY on the output grid)
    // T2:     R[ci][co][t] = sum_z X[ci][z] dY[co][2 z + d - 1]  (A = X on the coarse input grid)
    const bool t2 = mode == FE_NN_T2;
    const float *A = t2 ? d_x : d_dy, *B = t2 ? d_dy : d_x;
    const int ca = t2 ? cin : cout, cb = t2 ? cout : cin;
    const int *da = t2 ? dims_in : dims_out, *dbv = t2 ? dims_out : dims_in;
    const int stride = mode == FE_NN_S1 ? 1 : 2;
    size_t need = 0;
    int total_splits = 1;
    fe_status st = fe_nn_corr_workspace(stride, ca, da, cb, &need, &total_splits);
    if (st != FE_OK) return st;
    if (work_bytes < need) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const CorrShape cs = corr_shape(stride, ca, cb);
    const int split = total_splits / (cs.zs > 32 ? cs.zs / 32 : 1);
    dim3 grid(split, ((ca + 4 * cs.ag - 1) / (4 * cs.ag)) * ((cb + cs.bt - 1) / cs.bt));
    if (stride == 1) k_corr4<1><<<grid, kNnThreads, 0, s>>>(A, ca, dims_of(da), B, cb, dims_of(dbv), d_work, split, cs);
    else k_corr4<2><<<grid, kNnThreads, 0, s>>>(A, ca, dims_of(da), B, cb, dims_of(dbv), d_work, split, cs);
    FE_TRY_LAUNCH();
    k_corr_reduce<<<(ca * cb * 27 + 31) / 32, kNnThreads, 0, s>>>(d_work, total_splits, ca, cb, t2 ? 0 : 1, d_dw);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_channel_sum(const float *d_dy, int c, const int *dims, float *d_db, fe_stream_t stream) {
    if (!d_dy || !d_db || c < 1 || !dims_ok(dims)) return FE_ERR_ARG;
    const size_t plane = (size_t)dims[0] * dims[1] * dims[2];
    k_channel_sum<<<c * kSumCluster, kSumThreads, 0, (cudaStream_t)stream>>>(d_dy, plane, d_db);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_pack_weights(const float *d_w, int cin, int cout, int transpose, int flip,
                             void *d_outv, fe_stream_t stream) {
    __nv_bfloat16 *d_out = (__nv_bfloat16 *)d_outv;
    if (!d_w || !d_out || cin < 1 || cout < 1) return FE_ERR_ARG;
    k_pack_weights<<<grid1((size_t)cin * 27 * cout), kNnThreads, 0, (cudaStream_t)stream>>>(
        d_w, cin, cout, transpose, flip, d_out);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_relu_bwd(const float *d_y, float *d_dy, size_t n, fe_stream_t stream) {
    if (!d_y || !d_dy) return FE_ERR_ARG;
    if (n == 0) return FE_OK;
    k_relu_bwd<<<grid1(n), kNnThreads, 0, (cudaStream_t)stream>>>(d_y, d_dy, n);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_axpy(float a, const float *d_x, float *d_y, size_t n, fe_stream_t stream) {
    if (!d_x || !d_y) return FE_ERR_ARG;
    if (n == 0) return FE_OK;
    k_axpy<<<grid1(n), kNnThreads, 0, (cudaStream_t)stream>>>(a, d_x, d_y, n);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_head(const float *d_h, int c, const int *dims, const void *d_wv, const float *d_b,
                     float *d_out, fe_stream_t stream) {
    const __nv_bfloat16 *d_w = (const __nv_bfloat16 *)d_wv;
    if (!d_h || !d_w || !d_b || !d_out || c < 1 || !dims_ok(dims)) return FE_ERR_ARG;
    const size_t plane = (size_t)dims[0] * dims[1] * dims[2];
    k_head_fwd<<<grid1(plane), kNnThreads, 0, (cudaStream_t)stream>>>(d_h, c, plane, d_w, d_b, d_out);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_head_bwd(const float *d_h, int c, const int *dims, const void *d_wv,
                         const float *d_dout, float *d_dh, float *d_dw, float *d_db, float *d_work,
                         size_t work_bytes, fe_stream_t stream) {
    const __nv_bfloat16 *d_w = (const __nv_bfloat16 *)d_wv;
    if (!d_h || !d_w || !d_dout || !d_dh || !d_dw || !d_db || !d_work || c < 1 || !dims_ok(dims))
        return FE_ERR_ARG;
    const size_t plane = (size_t)dims[0] * dims[1] * dims[2];
    const int nb = 64;
    if (work_bytes < (size_t)(c + 1) * nb * sizeof(float)) return FE_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    k_head_bwd_data<<<grid1((size_t)c * plane), kNnThreads, 0, s>>>(d_dout, c, plane, d_w, d_dh);
    FE_TRY_LAUNCH();
    k_head_bwd_weight<<<dim3(nb, c), kNnThreads, 0, s>>>(d_h, d_dout, plane, d_work);
    FE_TRY_LAUNCH();
    k_rows_sum<<<1, 64, 0, s>>>(d_work, c, nb, d_dw);
    FE_TRY_LAUNCH();
    k_channel_sum<<<kSumCluster, kSumThreads, 0, s>>>(d_dout, plane, d_db);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_mse(const float *d_pred, const float *d_target, const uint8_t *d_bc_flag, size_t n,
                    float scale, float *d_dpred, float *d_loss_parts, int n_parts, fe_stream_t stream) {
    if (!d_pred || !d_target || !d_bc_flag || !d_dpred || !d_loss_parts || n_parts < 1) return FE_ERR_ARG;
    k_mse<<<n_parts, kNnThreads, 0, (cudaStream_t)stream>>>(d_pred, d_target, d_bc_flag, n, scale,
                                                             d_dpred, d_loss_parts);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_nn_adam(float *d_w, const float *d_g, float *d_m, float *d_v, size_t n, float lr_t,
                     float beta1, float beta2, float eps, fe_stream_t stream) {
    if (!d_w || !d_g || !d_m || !d_v) return FE_ERR_ARG;
    if (n == 0) return FE_OK;
    k_adam<<<grid1(n), kNnThreads, 0, (cudaStream_t)stream>>>(d_w, d_g, d_m, d_v, n, lr_t, beta1, beta2, eps);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_warmstart_input(const uint8_t *d_bc_flag, const double *d_bc_val, size_t n,
                             float *d_x, fe_stream_t stream) {
    if (!d_bc_flag || !d_bc_val || !d_x) return FE_ERR_ARG;
    k_ws_input<<<grid1(n), kNnThreads, 0, (cudaStream_t)stream>>>(d_bc_flag, d_bc_val, n, d_x);
    FE_TRY_LAUNCH();
    return FE_OK;
}

fe_status fe_warmstart_output(const float *d_pred, const uint8_t *d_bc_flag, const double *d_bc_val,
                              size_t n, double *d_x0, fe_stream_t stream) {
    if (!d_pred || !d_bc_flag || !d_bc_val || !d_x0) return FE_ERR_ARG;
    k_ws_output<<<grid1(n), kNnThreads, 0, (cudaStream_t)stream>>>(d_pred, d_bc_flag, d_bc_val, n, d_x0);
    FE_TRY_LAUNCH();
    return FE_OK;
}

}  // extern "C"
