// fe_warmstart.cu -- one call for the warm-start inference: boundary data of a
// mesh in, CG start vector out, through the 4-level encoder-decoder whose
// weights come in one blob.  Host-side orchestration of the network kernels
// (fe_nn.cu, fe_nn_tc.cu); allocates nothing.
//
// Network (levels l = 0..3 with n_l = (n_0 - 1) / 2^l + 1 nodes per axis,
// channels c0..c3; every conv 3x3x3 with bias):
//   e0 = relu(S1(x))          d1 = relu(S2(e0))   e1 = relu(S1(d1))
//   d2 = relu(S2(e1))         e2 = relu(S1(d2))   d3 = relu(S2(e2))  e3 = relu(S1(d3))
//   s2 = relu(T2(e3) + e2)    f2 = relu(S1(s2))
//   s1 = relu(T2(f2) + e1)    f1 = relu(S1(s1))
//   s0 = relu(T2(f1) + e0)    f0 = relu(S1(s0))
//   pred = head(f0) (1x1x1), x0 = bc_val on boundary nodes, pred inside.
#include <cstdint>

#include "fe_common.cuh"

namespace fe {

struct WsLayer {
    int mode, cin, cout, lin, lout;
};

// layer order of the blob: e0 d1 e1 d2 e2 d3 e3 u2 f2 u1 f1 u0 f0
static void ws_layers(const int *c, WsLayer *L) {
    const WsLayer t[13] = {{FE_NN_S1, 2, c[0], 0, 0},    {FE_NN_S2, c[0], c[1], 0, 1},
                           {FE_NN_S1, c[1], c[1], 1, 1}, {FE_NN_S2, c[1], c[2], 1, 2},
                           {FE_NN_S1, c[2], c[2], 2, 2}, {FE_NN_S2, c[2], c[3], 2, 3},
                           {FE_NN_S1, c[3], c[3], 3, 3}, {FE_NN_T2, c[3], c[2], 3, 2},
                           {FE_NN_S1, c[2], c[2], 2, 2}, {FE_NN_T2, c[2], c[1], 2, 1},
                           {FE_NN_S1, c[1], c[1], 1, 1}, {FE_NN_T2, c[1], c[0], 1, 0},
                           {FE_NN_S1, c[0], c[0], 0, 0}};
    for (int i = 0; i < 13; ++i) L[i] = t[i];
}

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

static bool ws_tc_ok(const WsLayer &l) {
    return (l.cout == 16 || l.cout == 32 || l.cout == 64) && l.cin >= 16;
}

// Blob: per layer bias FP32 [cout] then weights BF16 [cin][27][cout]; then the
// head weights BF16 [c0] and bias FP32 [1]; every section 256-byte aligned.
static size_t ws_blob_offsets(const int *c, size_t *off) {
    WsLayer L[13];
    ws_layers(c, L);
    size_t o = 0;
    for (int i = 0; i < 13; ++i) {
        off[2 * i] = o;
        o += al256((size_t)L[i].cout * 4);
        off[2 * i + 1] = o;
        o += al256((size_t)L[i].cin * 27 * L[i].cout * 2);
    }
    off[26] = o;
    o += al256((size_t)c[0] * 2);
    off[27] = o;
    o += al256(4);
    return o;
}

struct WsWork {
    size_t x_in, vol[15], pred, img[13], bf16i, total;
};

// activation buffers: x_in, e0 d1 e1 d2 e2 d3 e3 s2 f2 s1 f1 s0 f0 (13 volumes), pred; tensor-core images
static bool ws_work_layout(int n0, const int *c, WsWork *w) {
    if (n0 < 9 || (n0 - 1) % 8 != 0) return false;
    size_t nl[4];
    for (int l = 0; l < 4; ++l) {
        const size_t d = (size_t)((n0 - 1) >> l) + 1;
        nl[l] = d * d * d;
    }
    const int vc[13] = {c[0], c[1], c[1], c[2], c[2], c[3], c[3], c[2], c[2], c[1], c[1], c[0], c[0]};
    const int vl[13] = {0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
    size_t o = 0;
    w->x_in = o;
    o += al256(2 * nl[0] * 4);
    for (int i = 0; i < 13; ++i) {
        w->vol[i] = o;
        o += al256((size_t)vc[i] * nl[vl[i]] * 4);
    }
    w->pred = o;
    o += al256(nl[0] * 4);
    WsLayer L[13];
    ws_layers(c, L);
    size_t b16 = 0;   // largest BF16 interleaved layer input
    for (int i = 0; i < 13; ++i) {
        w->img[i] = o;
        if (ws_tc_ok(L[i])) {
            o += al256((size_t)((L[i].cin + 15) / 16) * 27 * 2 * L[i].cout * 16);
            const size_t need = (size_t)((L[i].cin + 7) / 8) * nl[L[i].lin] * 16;
            if (need > b16) b16 = need;
        }
    }
    w->bf16i = o;
    o += al256(b16);
    w->total = o;
    return true;
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_warmstart_blob_layout(const int *h_channels, size_t *h_offsets, size_t *h_bytes) {
    if (!h_channels || !h_bytes) return FE_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (h_channels[i] < 1) return FE_ERR_ARG;
    size_t off[28];
    *h_bytes = ws_blob_offsets(h_channels, off);
    if (h_offsets)
        for (int i = 0; i < 28; ++i) h_offsets[i] = off[i];
    return FE_OK;
}

fe_status fe_warmstart_workspace(int n_nodes, const int *h_channels, size_t *h_bytes) {
    if (!h_channels || !h_bytes) return FE_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (h_channels[i] < 1) return FE_ERR_ARG;
    WsWork w;
    if (!ws_work_layout(n_nodes, h_channels, &w)) return FE_ERR_ARG;
    *h_bytes = w.total;
    return FE_OK;
}

fe_status fe_warmstart_infer(int n_nodes, const int *h_channels, const void *d_blob, const uint8_t *d_bc_flag,
                             const double *d_bc_val, double *d_x0, void *d_work, size_t work_bytes,
                             int tensor_cores, fe_stream_t stream) {
    if (!h_channels || !d_blob || !d_bc_flag || !d_bc_val || !d_x0 || !d_work) return FE_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (h_channels[i] < 1) return FE_ERR_ARG;
    if (!aligned(d_blob, 256) || !aligned(d_work, 256)) return FE_ERR_ARG;
    WsWork w;
    if (!ws_work_layout(n_nodes, h_channels, &w)) return FE_ERR_ARG;
    if (work_bytes < w.total) return FE_ERR_WORKSPACE;
    size_t off[28];
    ws_blob_offsets(h_channels, off);
    WsLayer L[13];
    ws_layers(h_channels, L);
    const unsigned char *blob = (const unsigned char *)d_blob;
    unsigned char *ws = (unsigned char *)d_work;
    int dims[4][3];
    for (int l = 0; l < 4; ++l) dims[l][0] = dims[l][1] = dims[l][2] = ((n_nodes - 1) >> l) + 1;
    const size_t n0 = (size_t)n_nodes * n_nodes * n_nodes;
    auto vol = [&](int i) { return (float *)(ws + w.vol[i]); };
    auto bias = [&](int i) { return (const float *)(blob + off[2 * i]); };
    auto wts = [&](int i) { return (const void *)(blob + off[2 * i + 1]); };
    fe_status st;
#define WS_TRY(call)           \
    do {                       \
        st = (call);           \
        if (st != FE_OK) return st; \
    } while (0)
    // tensor-core operand images of this blob's weights
    const bool tc = tensor_cores != 0;
    if (tc)
        for (int i = 0; i < 13; ++i)
            if (ws_tc_ok(L[i])) WS_TRY(fe_nn_pack_weights_mma(wts(i), L[i].cin, L[i].cout, ws + w.img[i], stream));
    // layer i: input `src`, output volume vol(i), ReLU if `relu`
    auto layer = [&](int i, const float *src, int relu) -> fe_status {
        const WsLayer &l = L[i];
        float *dst = vol(i);
        if (tc && ws_tc_ok(l)) {
            // BF16 interleaved copy of the input, staged by TMA in the conv
            const fe_status cs = fe_nn_to_bf16i(src, l.cin, dims[l.lin], ws + w.bf16i, stream);
            if (cs != FE_OK) return cs;
            return fe_nn_conv3d_tc_bf16i(l.mode, ws + w.bf16i, l.cin, dims[l.lin], ws + w.img[i], bias(i), dst,
                                         l.cout, dims[l.lout], relu, stream);
        }
        return fe_nn_conv3d(l.mode, src, l.cin, dims[l.lin], wts(i), bias(i), dst, l.cout, dims[l.lout], relu,
                            stream);
    };
    auto nvox = [&](int i) {
        const size_t d = (size_t)dims[L[i].lout][0];
        return (size_t)L[i].cout * d * d * d;
    };
    float *x_in = (float *)(ws + w.x_in);
    WS_TRY(fe_warmstart_input(d_bc_flag, d_bc_val, n0, x_in, stream));
    WS_TRY(layer(0, x_in, 1));      // e0
    for (int i = 1; i <= 6; ++i) WS_TRY(layer(i, vol(i - 1), 1));   // d1 e1 d2 e2 d3 e3
    // decoder: s = relu(T2(.) + skip), f = relu(S1(s)); skips e2 (4), e1 (2), e0 (0)
    const int up[3] = {7, 9, 11}, skip[3] = {4, 2, 0};
    const float *src = vol(6);
    for (int k = 0; k < 3; ++k) {
        const int u = up[k];
        WS_TRY(layer(u, src, 0));
        WS_TRY(fe_nn_axpy(1.0f, vol(skip[k]), vol(u), nvox(u), stream));
        WS_TRY(fe_nn_relu_bwd(vol(u), vol(u), nvox(u), stream));
        WS_TRY(layer(u + 1, vol(u), 1));
        src = vol(u + 1);
    }
    float *pred = (float *)(ws + w.pred);
    WS_TRY(fe_nn_head(vol(12), h_channels[0], dims[0], blob + off[26], (const float *)(blob + off[27]), pred,
                      stream));
    WS_TRY(fe_warmstart_output(pred, d_bc_flag, d_bc_val, n0, d_x0, stream));
#undef WS_TRY
    return FE_OK;
}

}  // extern "C"
