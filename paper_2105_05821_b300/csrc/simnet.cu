// simnet.cu -- the C ABI of libsimnet (include/simnet.h): context, weights,
// workspaces and the lock-step simulation loop of Sec. 3.3, replayed as CUDA
// graphs of whole steps (gather -> conv GEMMs -> FC1 -> head + queue update).
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_fp16.h>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "ctx.cuh"
#include "tc_gemm.cuh"

using namespace simnet;

static constexpr int kGraphSteps = 16;

// Read-only view of a context's FP32 weights for entry points in other files.
namespace simnet {
bool ctx_fp32_view(const simnet_ctx *c, CtxFp32View &v) {
    if (!c || !c->has_weights || c->cfg.precision != SIMNET_FP32 || c->residual) return false;
    v.window = c->cfg.window;
    v.hidden = c->cfg.fc_hidden;
    v.n_layers = c->n_layers;
    for (int l = 0; l < c->n_layers; l++) v.layer[l] = c->layer[l];
    v.w2 = c->w2;
    v.b2 = c->b2;
    v.n_out = c->n_out;
    v.device = c->device;
    return true;
}
void ctx_set_error(simnet_ctx *c, const char *msg) {
    if (c) c->err = msg;
}
}  // namespace simnet

static size_t elem_size(int prec) { return prec == SIMNET_FP32 ? 4 : prec == SIMNET_BF16 ? 2 : 1; }

extern "C" int32_t simnet_abi_version(void) { return SIMNET_ABI_VERSION; }

extern "C" const char *simnet_last_error(const simnet_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" int64_t simnet_weight_count(const simnet_ctx *c) { return c ? c->n_weights : -1; }

extern "C" simnet_status simnet_init(const simnet_config *cfg, simnet_ctx **out) {
    if (!cfg || !out) return SIMNET_EINVAL;
    *out = nullptr;
    const simnet_config &k = *cfg;
    if (k.window < 2 || k.window > 256 || k.n_conv < 1 || k.n_conv > kMaxConv ||
        ((k.window >> k.n_conv) << k.n_conv) != k.window ||
        !(k.conv_channels == 64 || k.conv_channels == 128 || k.conv_channels == 256) || k.fc_hidden < 64 ||
        k.fc_hidden > 2048 || k.fc_hidden % 64 != 0 || k.retire_width < 1 || k.retire_width > 255 ||
        k.precision < SIMNET_FP32 || k.precision > SIMNET_FP8_E4M3)
        return SIMNET_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return SIMNET_ECUDA;
    simnet_ctx *c = new simnet_ctx();
    c->cfg = k;
    if (c->cfg.spin_limit_ns <= 0) c->cfg.spin_limit_ns = 2000000000LL;
    c->pdl = (k.flags & SIMNET_FLAG_NO_PDL) == 0;
    cudaGetDevice(&c->device);
    c->cap = k.window - 1;
    c->rows_n = k.window >> k.n_conv;
    c->fc1_in = c->rows_n * k.conv_channels;
    c->hybrid = (k.flags & SIMNET_FLAG_HYBRID_HEAD) != 0;
    c->store_queue = (k.flags & SIMNET_FLAG_STORE_QUEUE) != 0;
    c->n_lat = c->store_queue ? 3 : 2;
    c->n_out = (c->hybrid ? 11 : 1) * c->n_lat;
    c->residual = (k.flags & SIMNET_FLAG_RESIDUAL) != 0;
    c->n_blocks = c->residual ? k.n_conv : 0;
    c->n_layers = c->residual ? 3 * k.n_conv + 1 : k.n_conv + 1;   // GEMMs: 3 per residual block, + FC1
    if (c->residual && k.precision == SIMNET_FP8_E4M3) {
        delete c;
        return SIMNET_EUNSUPPORTED;
    }
    int64_t n = 0, cin = kNF;
    for (int l = 0; l < k.n_conv; l++) {
        n += (int64_t)k.conv_channels * cin * 2 + k.conv_channels;
        if (c->residual)   // pointwise conv + bias, projection shortcut
            n += (int64_t)k.conv_channels * k.conv_channels + k.conv_channels + (int64_t)k.conv_channels * cin * 2;
        cin = k.conv_channels;
    }
    n += (int64_t)c->fc1_in * k.fc_hidden + k.fc_hidden + (int64_t)c->n_out * k.fc_hidden + c->n_out;
    c->n_weights = n;
    for (int l = 0; l < c->n_layers; l++) {
        GemmLayer &g = c->layer[l];
        const bool fc1 = l == c->n_layers - 1;
        const int blk = c->residual ? l / 3 : l, part = c->residual ? l % 3 : 0;
        g.relu = 1;
        if (fc1) {
            g.m_mult = 1;
            g.K = c->fc1_in;
            g.N = k.fc_hidden;
            g.in_buf = k.n_conv == 0 ? kBufX : ((k.n_conv - 1) & 1) ? kBufAct1 : kBufAct0;
            g.out_buf = kBufH1;
            g.kind = k.n_conv;
            continue;
        }
        const int in = blk == 0 ? kBufX : ((blk - 1) & 1) ? kBufAct1 : kBufAct0;
        const int out = (blk & 1) ? kBufAct1 : kBufAct0;
        g.m_mult = k.window >> (blk + 1);
        g.N = k.conv_channels;
        g.kind = blk;
        if (part == 2) {   // residual block: pointwise conv of the branch, plus the shortcut
            g.K = k.conv_channels;
            g.in_buf = kBufTmpA;
            g.out_buf = out;
            g.res_buf = kBufTmpS;
        } else {           // conv layer, or a block's conv (branch) / projection (shortcut)
            g.K = blk == 0 ? 2 * kNFP : 2 * k.conv_channels;
            g.in_buf = in;
            g.out_buf = !c->residual ? out : part == 0 ? kBufTmpA : kBufTmpS;
            g.relu = part == 1 ? 0 : 1;
        }
    }
    *out = c;
    return SIMNET_OK;
}

static void free_workspace(simnet_ctx *c) {
    void *bufs[] = {c->X, c->act[0], c->act[1], c->h1, c->tick, c->pos, c->qstart, c->qlen, c->evict,
                    c->active, c->n_active, c->status, c->cnt, c->ring, c->totals, c->d_args, c->cyc,
                    c->mstart, c->mlen, c->mring, c->tmpA, c->tmpS};
    for (void *p : bufs)
        if (p) cudaFree(p);
    c->X = c->act[0] = c->act[1] = c->tmpA = c->tmpS = nullptr;
    c->h1 = nullptr;
    c->tick = c->pos = c->qstart = c->qlen = c->evict = c->active = c->n_active = c->status = c->cnt = nullptr;
    c->ring = nullptr;
    c->mstart = c->mlen = nullptr;
    c->mring = nullptr;
    c->cyc = nullptr;
    c->totals = nullptr;
    c->d_args = nullptr;
    c->ws_B = 0;
    for (auto &q : c->pbuf)
        if (q) { cudaFree(q); q = nullptr; }
    c->pbuf_B = 0;
    for (auto &g : c->gexec)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    c->g_B = -1;
}

extern "C" void simnet_destroy(simnet_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_workspace(c);
    TrainState &t = c->tr;
    for (int l = 0; l < kMaxGemm; l++) {
        void *tb[] = {t.gW[l], t.gb[l], t.mW[l], t.vW[l], t.mb[l], t.vb[l], t.Y[l], t.Yb[l]};
        for (void *q : tb)
            if (q) cudaFree(q);
        if (c->W32[l] && (void *)c->W32[l] != c->Wl[l]) cudaFree(c->W32[l]);
    }
    {
        void *tb[] = {t.gw2, t.gb2, t.mw2, t.vw2, t.mb2, t.vb2, t.X, t.dA, t.dB, t.z, t.dz, t.loss,
                      t.Xb, t.dHb, t.dYb[0], t.dYb[1], t.wpart, t.colpart};
        for (void *q : tb)
            if (q) cudaFree(q);
    }
    for (int l = 0; l < kMaxGemm; l++) {
        if (c->Wl[l]) cudaFree(c->Wl[l]);
        if (c->bias[l]) cudaFree(c->bias[l]);
        if (c->wscale[l]) cudaFree(c->wscale[l]);
        if (c->oscale[l]) cudaFree(c->oscale[l]);
    }
    if (c->w2) cudaFree(c->w2);
    if (c->b2) cudaFree(c->b2);
    if (c->layer_const) cudaFree(c->layer_const);
    if (c->h_args) cudaFreeHost(c->h_args);
    if (c->h_offsets) cudaFreeHost(c->h_offsets);
    if (c->h_totals) cudaFreeHost(c->h_totals);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->args_ev) cudaEventDestroy(c->args_ev);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    if (c->bar) cudaFree(c->bar);
    if (c->bar_abort) cudaFree(c->bar_abort);
    if (c->phase_ns) cudaFree(c->phase_ns);
    if (c->phase_n) cudaFree(c->phase_n);
    if (c->fc1_const) cudaFree(c->fc1_const);
    if (c->ext) cudaFree(c->ext);
    delete c;
}

template <typename T>
static simnet_status upload(simnet_ctx *c, void **dst, const std::vector<T> &v) {
    if (*dst) { cudaFree(*dst); *dst = nullptr; }
    CK(cudaMalloc(dst, v.size() * sizeof(T)));
    CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SIMNET_OK;
}

// Synthetic context rows for the FP8 calibration pass: a current instruction and
// a random number of context rows with the feature encoding's value ranges
// (one-hots, register ids / 32, flags, residence and execution latency / 64).
static void synthetic_windows(int n, int W, std::vector<float> &x) {
    x.assign((size_t)n * W * kNFP, 0.f);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto rnd = [&st]() {  // xorshift64*
        st ^= st >> 12;
        st ^= st << 25;
        st ^= st >> 27;
        return (uint32_t)((st * 0x2545F4914F6CDD1Dull) >> 32);
    };
    auto uni = [&]() { return (rnd() >> 8) * (1.0f / 16777216.0f); };
    for (int i = 0; i < n; i++) {
        const int len = (int)(rnd() % (uint32_t)W);
        for (int r = 0; r <= len && r < W; r++) {
            float *row = &x[((size_t)i * W + r) * kNFP];
            row[rnd() % 32] = 1.f;
            for (int j = 32; j < 35; j++) row[j] = (float)(rnd() % 32) / 32.f;
            row[35] = uni() < 0.25f;
            row[36] = uni() < 0.10f;
            row[37] = uni() < 0.15f;
            row[38 + rnd() % 3] = 1.f;
            row[41] = uni() < 0.05f;
            if (r > 0) {
                const float u = uni();
                row[42] = u * u * 4.f;           // residence up to 256 cycles, mostly short
                row[43] = (float)(rnd() % 64) / 64.f;
                for (int j = 45; j < 48; j++) row[j] = uni() < 0.03125f;
                row[48] = uni() < 0.1f;
            }
        }
    }
}

// FP8 activation scales: run the FP32 layers on synthetic rows and take each
// conv output channel's maximum (x2 margin) / 448, the e4m3 maximum.
static simnet_status calibrate_fp8(simnet_ctx *c, const std::vector<std::vector<float>> &Wg,
                                   const std::vector<std::vector<float>> &Bg, std::vector<std::vector<float>> &s_act) {
    const simnet_config &k = c->cfg;
    const int n = 512, W = k.window, C = k.conv_channels;
    std::vector<float> xh;
    synthetic_windows(n, W, xh);
    float *x = nullptr, *y[2] = {nullptr, nullptr}, *w = nullptr, *b = nullptr;
    int32_t *cnt = nullptr;
    unsigned *amax = nullptr;
    auto cleanup = [&]() {
        cudaFree(x); cudaFree(y[0]); cudaFree(y[1]); cudaFree(w); cudaFree(b); cudaFree(cnt); cudaFree(amax);
    };
    const size_t ybytes = (size_t)n * (W / 2) * C * sizeof(float);
    size_t wmax = 0;
    for (int l = 0; l < k.n_conv; l++) wmax = std::max(wmax, Wg[l].size());
    if (cudaMalloc(&x, xh.size() * 4) != cudaSuccess || cudaMalloc(&y[0], ybytes) != cudaSuccess ||
        cudaMalloc(&y[1], ybytes) != cudaSuccess || cudaMalloc(&w, wmax * 4) != cudaSuccess ||
        cudaMalloc(&b, (size_t)C * 4) != cudaSuccess || cudaMalloc(&cnt, 4) != cudaSuccess ||
        cudaMalloc(&amax, (size_t)C * 4) != cudaSuccess) {
        cleanup();
        return fail(c, SIMNET_ENOMEM, "FP8 calibration: allocation failed");
    }
    cudaMemcpy(x, xh.data(), xh.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(cnt, &n, 4, cudaMemcpyHostToDevice);
    s_act.assign(k.n_conv, std::vector<float>(C, 1.f));
    const float *in = x;
    for (int l = 0; l < k.n_conv; l++) {
        const GemmLayer &g = c->layer[l];
        cudaMemcpy(w, Wg[l].data(), Wg[l].size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(b, Bg[l].data(), (size_t)C * 4, cudaMemcpyHostToDevice);
        launch_gemm_f32(in, w, b, y[l & 1], cnt, g.m_mult, n * g.m_mult, g.N, g.K, 1, 0);
        cudaMemset(amax, 0, (size_t)C * 4);
        launch_channel_amax(y[l & 1], (int64_t)n * g.m_mult, C, amax, 0);
        std::vector<unsigned> am(C);
        if (cudaMemcpy(am.data(), amax, (size_t)C * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cleanup();
            return fail(c, SIMNET_ECUDA, "FP8 calibration failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        for (int ch = 0; ch < C; ch++) {
            float m;
            memcpy(&m, &am[ch], 4);
            s_act[l][ch] = m > 0.f ? 2.f * m / 448.f : 1.f;
        }
        in = y[l & 1];
    }
    cleanup();
    return SIMNET_OK;
}

// Re-lay the canonical PyTorch-shaped weights into GEMM operands [N][K]:
// conv k: K index = t * Cin_pad + ci for kernel tap t of input channel ci
// (rows 2l and 2l+1 of the input are adjacent, so a conv output row is one dot
// product with a contiguous 2*Cin_pad slice); FC1: K index = l * C + c for the
// canonical input index c * L_n + l (the device flatten keeps rows outermost).
// Rows past every queue are zero features, so every conv layer maps them to
// one constant row; FC1 then sees that row at each padded position.  Follow
// the constant through the layers with the stored precision's rounding and
// tabulate S[e] = sum over positions l >= e of FC1's weights times it.
simnet_status build_fc1_const(simnet_ctx *c, const std::vector<std::vector<float>> &Bg,
                              const std::vector<std::vector<float>> &Wdeq,
                              const std::vector<std::vector<float>> &osc) {
    const simnet_config &k = c->cfg;
    const int C = k.conv_channels, H = k.fc_hidden, Ln = c->rows_n;
    auto quant = [&](int l, int n, double x) -> double {
        if (k.precision == SIMNET_BF16) return (double)__bfloat162float(__float2bfloat16_rn((float)x));
        const float o = osc[l][n];
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8((float)x * o, __NV_SATFINITE, __NV_E4M3);
        return (double)__half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))) / o;
    };
    // each layer's constant output row as the kernels store it (BF16, or the FP8 byte
    // of value * requant multiplier), for the persistent kernel's per-layer extent
    std::vector<float> lc((size_t)(c->n_layers - 1) * C, 0.f);
    auto keep = [&](int l, const std::vector<double> &v) {
        for (int n = 0; n < C; n++)
            lc[(size_t)l * C + n] = k.precision == SIMNET_BF16 ? (float)v[n] : (float)(v[n] * osc[l][n]);
    };
    std::vector<double> cst(kNFP, 0.0);
    int cin_pad = kNFP;
    // a k=2 / stride-2 GEMM layer on a pair of constant rows (bias, optional ReLU, stored rounding)
    auto pair_layer = [&](int l, int cp, bool relu) {
        const int K = c->layer[l].K;
        std::vector<double> nxt(C);
        for (int n = 0; n < C; n++) {
            double acc = Bg[l][n];
            for (int kk = 0; kk < K; kk++) acc += (double)Wdeq[l][(size_t)n * K + kk] * cst[kk % cp];
            nxt[n] = quant(l, n, relu && acc < 0.0 ? 0.0 : acc);
        }
        keep(l, nxt);
        return nxt;
    };
    for (int b = 0; b < k.n_conv; b++) {
        if (!c->residual) {
            cst = pair_layer(b, cin_pad, true);
        } else {   // residual block: branch a, shortcut s, then ReLU(pw(a) + s)
            const std::vector<double> a_c = pair_layer(3 * b, cin_pad, true), s_c = pair_layer(3 * b + 1, cin_pad, false);
            const int l = 3 * b + 2;
            std::vector<double> nxt(C);
            for (int n = 0; n < C; n++) {
                double acc = Bg[l][n] + s_c[n];
                for (int j = 0; j < C; j++) acc += (double)Wdeq[l][(size_t)n * C + j] * a_c[j];
                nxt[n] = quant(l, n, acc > 0.0 ? acc : 0.0);
            }
            keep(l, nxt);
            cst = nxt;
        }
        cin_pad = C;
    }
    simnet_status st0 = upload(c, (void **)&c->layer_const, lc);
    if (st0 != SIMNET_OK) return st0;
    const int L = c->n_layers - 1, K1 = c->fc1_in;
    std::vector<float> S((size_t)(Ln + 1) * H, 0.f);
    for (int n = 0; n < H; n++) {
        double run = 0.0;
        for (int e = Ln - 1; e >= 0; e--) {
            for (int ch = 0; ch < C; ch++) run += (double)Wdeq[L][(size_t)n * K1 + (size_t)e * C + ch] * cst[ch];
            S[(size_t)e * H + n] = (float)run;
        }
    }
    return upload(c, (void **)&c->fc1_const, S);
}

// BF16 contexts whose FP32 masters changed on the device (training steps, new
// device weights): the kernels use bf16(W32), so the table follows from those.
simnet_status refresh_fc1_const(simnet_ctx *c) {
    if (c->cfg.precision != SIMNET_BF16) return fail(c, SIMNET_ESTATE, "padding table: only BF16 weights change on the device");
    CK(cudaDeviceSynchronize());
    std::vector<std::vector<float>> Bg(c->n_layers), Wdeq(c->n_layers), osc;
    for (int l = 0; l < c->n_layers; l++) {
        const GemmLayer &g = c->layer[l];
        Wdeq[l].resize((size_t)g.N * g.K);
        Bg[l].resize(g.N);
        CK(cudaMemcpy(Wdeq[l].data(), c->W32[l], Wdeq[l].size() * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(Bg[l].data(), c->bias[l], (size_t)g.N * 4, cudaMemcpyDeviceToHost));
        for (float &w : Wdeq[l]) w = __bfloat162float(__float2bfloat16_rn(w));
    }
    simnet_status st = build_fc1_const(c, Bg, Wdeq, osc);
    if (st == SIMNET_OK) c->const_stale = false;
    return st;
}

// Fingerprint of the FP32 weights in canonical order (the loaded blob's, or of
// the current device masters after on-device updates).
uint64_t weights_fingerprint(simnet_ctx *c) {
    if (c->weights_fp_dirty) {
        std::vector<float> blob((size_t)c->n_weights);
        if (simnet_get_weights(c, blob.data()) != SIMNET_OK) return 0;
        c->weights_fp = fnv1a(blob.data(), blob.size() * sizeof(float));
        c->weights_fp_dirty = false;
    }
    return c->weights_fp;
}

extern "C" simnet_status simnet_load_weights(simnet_ctx *c, const float *blob, int64_t n_values) {
    if (!c) return SIMNET_EINVAL;
    if (!blob) return fail(c, SIMNET_EINVAL, "load_weights: blob is NULL");
    if (n_values != c->n_weights)
        return fail(c, SIMNET_EINVAL, "load_weights: got %lld values, config needs %lld", (long long)n_values,
                    (long long)c->n_weights);
    const simnet_config &k = c->cfg;
    const int C = k.conv_channels, H = k.fc_hidden, Ln = c->rows_n;
    std::vector<std::vector<float>> Wg(c->n_layers), Bg(c->n_layers);
    const float *p = blob;
    int cin = kNF;
    // a k=2 / stride-2 conv [C][cin][2] as a GEMM [C][2 * cin_pad] (K = tap * cin_pad + channel)
    auto conv_gemm = [&](std::vector<float> &dst, int cin_pad) {
        const int K = 2 * cin_pad;
        dst.assign((size_t)C * K, 0.f);
        for (int co = 0; co < C; co++)
            for (int ci = 0; ci < cin; ci++)
                for (int t = 0; t < 2; t++) dst[(size_t)co * K + t * cin_pad + ci] = p[((size_t)co * cin + ci) * 2 + t];
        p += (size_t)C * cin * 2;
    };
    for (int b = 0; b < k.n_conv; b++) {
        const int cin_pad = b == 0 ? kNFP : C;
        const int l = c->residual ? 3 * b : b;
        conv_gemm(Wg[l], cin_pad);
        Bg[l].assign(p, p + C);
        p += C;
        if (c->residual) {   // pointwise conv [C][C][1] = GEMM [C][C]; then the bias-free projection
            Wg[l + 2].assign(p, p + (size_t)C * C);
            p += (size_t)C * C;
            Bg[l + 2].assign(p, p + C);
            p += C;
            conv_gemm(Wg[l + 1], cin_pad);
            Bg[l + 1].assign(C, 0.f);
        }
        cin = C;
    }
    {
        const int l = c->n_layers - 1, K = c->fc1_in;
        Wg[l].assign((size_t)H * K, 0.f);
        for (int h = 0; h < H; h++)
            for (int ch = 0; ch < C; ch++)
                for (int r = 0; r < Ln; r++) Wg[l][(size_t)h * K + r * C + ch] = p[(size_t)h * K + (size_t)ch * Ln + r];
        p += (size_t)H * K;
        Bg[l].assign(p, p + H);
        p += H;
    }
    const int NO = c->n_out;
    std::vector<float> w2(p, p + (size_t)NO * H), b2(p + (size_t)NO * H, p + (size_t)NO * H + NO);
    simnet_status st;
    std::vector<std::vector<float>> s_act;
    if (k.precision == SIMNET_FP8_E4M3 && (st = calibrate_fp8(c, Wg, Bg, s_act)) != SIMNET_OK) return st;
    // what the kernels multiply by, in true units (GEMM layout), and how each
    // layer's stored activations round: for the padding constants below
    std::vector<std::vector<float>> Wdeq(c->n_layers), osc(c->n_layers);
    for (int l = 0; l < c->n_layers; l++) {
        if (k.precision == SIMNET_FP8_E4M3) {
            // B[n][k] = W[n][k] * s_in[k] / s_w[n]: the input's per-channel scale folded
            // along K, a per-output-channel scale s_w taken back out in the epilogue,
            // which also divides by the next layer's input scale (oscale).
            const GemmLayer &g = c->layer[l];
            const int K = g.K, Nn = g.N, cin_pad = l == 0 ? kNFP : C;
            std::vector<float> sin(K, 1.f), sw(Nn), os(Nn);
            if (l > 0)
                for (int kk = 0; kk < K; kk++) sin[kk] = s_act[l - 1][kk % cin_pad];
            std::vector<__nv_fp8_storage_t> wq((size_t)Nn * K);
            for (int n = 0; n < Nn; n++) {
                float mx = 0.f;
                for (int kk = 0; kk < K; kk++) mx = fmaxf(mx, fabsf(Wg[l][(size_t)n * K + kk] * sin[kk]));
                sw[n] = mx > 0.f ? mx / 448.f : 1.f;
                for (int kk = 0; kk < K; kk++)
                    wq[(size_t)n * K + kk] =
                        __nv_cvt_float_to_fp8(Wg[l][(size_t)n * K + kk] * sin[kk] / sw[n], __NV_SATFINITE, __NV_E4M3);
                os[n] = l < k.n_conv ? 1.f / s_act[l][n] : 1.f;
            }
            Wdeq[l].resize(wq.size());
            for (int n = 0; n < Nn; n++)
                for (int kk = 0; kk < K; kk++) {
                    const __half_raw hr = __nv_cvt_fp8_to_halfraw(wq[(size_t)n * K + kk], __NV_E4M3);
                    Wdeq[l][(size_t)n * K + kk] = __half2float(__half(hr)) * sw[n] / sin[kk];
                }
            osc[l] = os;
            if ((st = upload(c, &c->Wl[l], wq)) != SIMNET_OK) return st;
            if ((st = upload(c, (void **)&c->wscale[l], sw)) != SIMNET_OK) return st;
            if (l < k.n_conv) {
                if ((st = upload(c, (void **)&c->oscale[l], os)) != SIMNET_OK) return st;
            } else if (c->oscale[l]) {
                cudaFree(c->oscale[l]);
                c->oscale[l] = nullptr;
            }
        } else if (k.precision == SIMNET_FP32) {
            if ((st = upload(c, &c->Wl[l], Wg[l])) != SIMNET_OK) return st;
            c->W32[l] = (float *)c->Wl[l];
        } else if (k.precision == SIMNET_BF16) {
            std::vector<__nv_bfloat16> wb(Wg[l].size());
            Wdeq[l].resize(wb.size());
            for (size_t i = 0; i < wb.size(); i++) {
                wb[i] = __float2bfloat16_rn(Wg[l][i]);
                Wdeq[l][i] = __bfloat162float(wb[i]);
            }
            if ((st = upload(c, &c->Wl[l], wb)) != SIMNET_OK) return st;
            if ((st = upload(c, (void **)&c->W32[l], Wg[l])) != SIMNET_OK) return st;
        }
        if ((st = upload(c, (void **)&c->bias[l], Bg[l])) != SIMNET_OK) return st;
        c->layer[l].B = c->Wl[l];
        c->layer[l].bias = c->bias[l];
        c->layer[l].scale = c->wscale[l];
        c->layer[l].oscale = c->oscale[l];
    }
    if ((st = upload(c, (void **)&c->w2, w2)) != SIMNET_OK) return st;
    if ((st = upload(c, (void **)&c->b2, b2)) != SIMNET_OK) return st;
    if (k.precision != SIMNET_FP32 && (st = build_fc1_const(c, Bg, Wdeq, osc)) != SIMNET_OK) return st;
    if (c->residual) c->blob_host.assign(blob, blob + n_values);
    c->weights_fp = fnv1a(blob, (size_t)n_values * sizeof(float));
    c->weights_fp_dirty = false;
    c->const_stale = false;
    c->has_weights = true;
    c->tr.plan_n = -1;   // the training GEMMs hold the old weight buffers
    if (c->tr.ready) {  // new weights: restart the optimiser
        TrainState &t = c->tr;
        t.step = 0;
        for (int l = 0; l < c->n_layers; l++) {
            const size_t wn = (size_t)c->layer[l].N * c->layer[l].K;
            cudaMemset(t.mW[l], 0, wn * 4);
            cudaMemset(t.vW[l], 0, wn * 4);
            cudaMemset(t.mb[l], 0, (size_t)c->layer[l].N * 4);
            cudaMemset(t.vb[l], 0, (size_t)c->layer[l].N * 4);
        }
        cudaMemset(t.mw2, 0, (size_t)c->n_out * k.fc_hidden * 4);
        cudaMemset(t.vw2, 0, (size_t)c->n_out * k.fc_hidden * 4);
        cudaMemset(t.mb2, 0, (size_t)c->n_out * 4);
        cudaMemset(t.vb2, 0, (size_t)c->n_out * 4);
    }
    for (auto &g : c->gexec)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    c->g_B = -1;
    return SIMNET_OK;
}

simnet_status ensure_workspace(simnet_ctx *c, int B) {
    if (B <= c->ws_B) return SIMNET_OK;
    CK(cudaDeviceSynchronize());
    free_workspace(c);
    c->sim_valid = false;
    const simnet_config &k = c->cfg;
    const size_t es = elem_size(k.precision);
    const size_t xb = (size_t)B * k.window * kNFP * es;
    const size_t ab = (size_t)B * std::max(k.window / 2, 2) * k.conv_channels * es;
    CK(cudaMalloc(&c->X, xb));
    CK(cudaMalloc(&c->act[0], ab));
    CK(cudaMalloc(&c->act[1], ab));
    if (c->residual) {
        CK(cudaMalloc(&c->tmpA, ab));
        CK(cudaMalloc(&c->tmpS, ab));
    }
    // FC2 partials: at most fc_hidden / 32 column blocks (64-wide tiles, two halves) x n_out per row
    const size_t h1n = std::max((size_t)k.fc_hidden, (size_t)(k.fc_hidden / 32) * c->n_out);
    CK(cudaMalloc(&c->h1, (size_t)B * h1n * sizeof(float)));
    CK(cudaMalloc(&c->tick, (size_t)B * 4));
    CK(cudaMalloc(&c->pos, (size_t)B * 4));
    CK(cudaMalloc(&c->qstart, (size_t)B * 4));
    CK(cudaMalloc(&c->qlen, (size_t)B * 4));
    CK(cudaMalloc(&c->evict, (size_t)B * 4));
    CK(cudaMalloc(&c->active, (size_t)B * 4));
    CK(cudaMalloc(&c->n_active, 4));
    CK(cudaMalloc(&c->status, 4));
    CK(cudaMalloc(&c->cnt, 4));
    CK(cudaMalloc(&c->ring, (size_t)B * c->cap * sizeof(uint64_t)));
    if (c->store_queue) {
        CK(cudaMalloc(&c->mstart, (size_t)B * 4));
        CK(cudaMalloc(&c->mlen, (size_t)B * 4));
        CK(cudaMalloc(&c->mring, (size_t)B * c->cap * sizeof(uint64_t)));
    }
    CK(cudaMalloc(&c->cyc, (size_t)B * sizeof(int64_t)));
    CK(cudaMalloc(&c->totals, 2 * sizeof(unsigned long long)));
    CK(cudaMalloc(&c->d_args, sizeof(StepArgs)));
    if (!c->bar) {
        CK(cudaMalloc(&c->bar, sizeof(unsigned)));
        CK(cudaMalloc(&c->bar_abort, sizeof(int)));
        CK(cudaMalloc(&c->phase_ns, 64 * sizeof(unsigned long long)));
        CK(cudaMalloc(&c->phase_n, SIMNET_KERNEL_KINDS * sizeof(unsigned long long)));
        CK(cudaMalloc(&c->ext, 4 * sizeof(int)));
    }
    if (!c->h_args) {
        CK(cudaMallocHost(&c->h_args, sizeof(StepArgs)));
        CK(cudaMallocHost(&c->h_totals, 2 * sizeof(unsigned long long)));
        CK(cudaMallocHost(&c->h_status, sizeof(int32_t)));
        CK(cudaEventCreateWithFlags(&c->args_ev, cudaEventDisableTiming));
        CK(cudaEventCreate(&c->ev0));
        CK(cudaEventCreate(&c->ev1));
        CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    }
    c->ws_B = B;
    return SIMNET_OK;
}

// The CNN on the batch already in c->X: conv GEMMs, then FC1 into c->h1.
// `count` is a device int of active rows-groups (sub-traces or windows).
// The CNN on the batch already in c->X: conv GEMMs, then FC1 with FC2 folded
// into its epilogue, leaving c->n_part partial sums per row in c->h1.
// Workspace buffer of a GemmBuf id.
static void *wsbuf(simnet_ctx *c, int id) {
    switch (id) {
        case kBufX: return c->X;
        case kBufAct0: return c->act[0];
        case kBufAct1: return c->act[1];
        case kBufTmpA: return c->tmpA;
        case kBufTmpS: return c->tmpS;
        case kBufH1: return c->h1;
        default: return nullptr;
    }
}

static void enqueue_cnn(simnet_ctx *c, const int32_t *count, int B, cudaStream_t s, bool pdl,
                        KTimer *kt = nullptr) {
    const simnet_config &k = c->cfg;
    for (int l = 0; l < c->n_layers; l++) {
        const GemmLayer &g = c->layer[l];
        if (kt) kt->begin(SIMNET_KERNEL_LAYER0 + g.kind);
        const bool last = l == c->n_layers - 1;
        const void *in = wsbuf(c, g.in_buf);
        void *out = wsbuf(c, g.out_buf);
        const int m_cap = B * g.m_mult;
        if (k.precision == SIMNET_FP32) {
            if (last)
                launch_gemm_f32_part((const float *)in, (const float *)g.B, g.bias, c->w2, (float *)out, B, count,
                                     g.m_mult, m_cap, g.N, g.K, g.relu, c->n_out, s, pdl);
            else
                launch_gemm_f32((const float *)in, (const float *)g.B, g.bias, (float *)out, count, g.m_mult, m_cap,
                                g.N, g.K, g.relu, s, pdl, (const float *)wsbuf(c, g.res_buf));
        } else {
            launch_tc_gemm(c->plan[l], g, count, c->w2, s);
        }
        if (kt) kt->end();
    }
}

static int launches_per_step(const simnet_ctx *c) { return c->n_layers + 1; }

// Context gather of every slot into c->X (first step, and after a compaction
// has moved sub-traces to new slots); other steps get their rows from the
// previous step's head/update kernel.
static void enqueue_gather(simnet_ctx *c, int B, cudaStream_t s, bool pdl, KTimer *kt = nullptr) {
    if (kt) kt->begin(SIMNET_KERNEL_GATHER);
    switch (c->cfg.precision) {
        case SIMNET_FP32: launch_gather<float>(c->d_args, (float *)c->X, B, c->cfg.window, s, pdl); break;
        case SIMNET_BF16:
            launch_gather<__nv_bfloat16>(c->d_args, (__nv_bfloat16 *)c->X, B, c->cfg.window, s, pdl);
            break;
        default: launch_gather<__nv_fp8_e4m3>(c->d_args, (__nv_fp8_e4m3 *)c->X, B, c->cfg.window, s, pdl); break;
    }
    if (kt) kt->end();
}

static void enqueue_step(simnet_ctx *c, int B, cudaStream_t s, bool pdl, KTimer *kt = nullptr) {
    enqueue_cnn(c, c->n_active, B, s, pdl, kt);
    if (kt) kt->begin(SIMNET_KERNEL_HEAD_UPDATE);
    const float *part = c->h1;
    const int NO = c->n_out;
    switch (c->cfg.precision) {
        case SIMNET_FP32:
            launch_head_update<float>(c->d_args, part, c->n_part, B, c->b2, (float *)c->X, B, NO, s, pdl);
            break;
        case SIMNET_BF16:
            launch_head_update<__nv_bfloat16>(c->d_args, part, c->n_part, B, c->b2, (__nv_bfloat16 *)c->X, B, NO, s,
                                              pdl);
            break;
        default:
            launch_head_update<__nv_fp8_e4m3>(c->d_args, part, c->n_part, B, c->b2, (__nv_fp8_e4m3 *)c->X, B, NO, s,
                                              pdl);
            break;
    }
    if (kt) kt->end();
}

static void enqueue_compact(simnet_ctx *c, int B, cudaStream_t s, bool pdl, KTimer *kt = nullptr) {
    if (kt) kt->begin(SIMNET_KERNEL_COMPACT);
    launch_compact(c->d_args, s, pdl);
    if (kt) kt->end();
    enqueue_gather(c, B, s, pdl, kt);
}

static simnet_status prepare_plans(simnet_ctx *c, int B, bool pdl) {
    const GemmLayer &fc1 = c->layer[c->n_layers - 1];
    if (c->cfg.precision == SIMNET_FP32) {
        c->n_part = gemm_f32_part_blocks(fc1.N);
        return SIMNET_OK;
    }
    for (int l = 0; l < c->n_layers; l++) {
        const GemmLayer &g = c->layer[l];
        const bool last = l == c->n_layers - 1;
        const void *in = wsbuf(c, g.in_buf);
        void *out = wsbuf(c, g.out_buf);
        std::string why;
        const int ok_kind = !last ? TC_OUT_ACT
                            : c->n_out == 3 ? TC_OUT_PART3
                            : c->n_out == 22 ? TC_OUT_PART_HYBRID
                            : c->n_out == 33 ? TC_OUT_PART33 : TC_OUT_PART;
        if (!make_tc_plan(c->plan[l], c->cfg.precision, in, g, out, ok_kind, B * g.m_mult,
                          c->cfg.spin_limit_ns, c->status, pdl, why, wsbuf(c, g.res_buf)))
            return fail(c, SIMNET_ECUDA, "tensor-core plan for layer %d: %s", l, why.c_str());
        if (c->tuned_B == B && c->tuned_bn[l] && c->tuned_bn[l] != c->plan[l].BN &&
            !retune_tc_plan(c->plan[l], g, c->tuned_bn[l], why))
            return fail(c, SIMNET_ECUDA, "tuned tile for layer %d: %s", l, why.c_str());
    }
    c->n_part = 2 * (fc1.N / c->plan[c->n_layers - 1].BN);   // two column halves per block
    return SIMNET_OK;
}

static simnet_status capture_graphs(simnet_ctx *c, int B, bool compact) {
    for (auto &g : c->gexec)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    for (int gi = 0; gi < 2; gi++) {
        const int steps = gi == 0 ? kGraphSteps : 1;
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < steps; i++) enqueue_step(c, B, c->cap_stream, c->pdl && i > 0);
        if (compact) enqueue_compact(c, B, c->cap_stream, c->pdl);
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (e != cudaSuccess) return fail(c, SIMNET_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec[gi], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(c, SIMNET_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    c->g_B = B;
    c->g_compact = compact;
    return SIMNET_OK;
}

extern "C" simnet_status simnet_simulate(simnet_ctx *c, const simnet_trace *t, int64_t *cycles_out,
                                         uint8_t *lat_log, float *pre_log, const uint8_t *lat_replay,
                                         simnet_stats *stats, void *stream) {
    return simnet_simulate_steps(c, t, cycles_out, lat_log, pre_log, lat_replay, -1, 0, stats, stream);
}

extern "C" simnet_status simnet_simulate_steps(simnet_ctx *c, const simnet_trace *t, int64_t *cycles_out,
                                               uint8_t *lat_log, float *pre_log, const uint8_t *lat_replay,
                                               int64_t max_steps, int32_t resume, simnet_stats *stats,
                                               void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!t || t->n_subtraces < 0 || t->n_instructions < 0 || (t->n_subtraces > 0 && !cycles_out))
        return fail(c, SIMNET_EINVAL, "simulate: null trace/cycles_out or negative sizes");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "simulate: no weights loaded");
    if (t->n_subtraces > 0 && (!t->offsets || (t->n_instructions > 0 && !t->records)))
        return fail(c, SIMNET_EINVAL, "simulate: null records/offsets");
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int B = t->n_subtraces;
    if (stats) memset(stats, 0, sizeof *stats);
    if (B == 0) return SIMNET_OK;

    // offsets -> host: validate and find the number of lock-step iterations
    if ((size_t)(B + 1) > c->h_offsets_cap) {
        if (c->h_offsets) cudaFreeHost(c->h_offsets);
        c->h_offsets = nullptr;
        CK(cudaMallocHost(&c->h_offsets, (size_t)(B + 1) * sizeof(int64_t)));
        c->h_offsets_cap = (size_t)B + 1;
    }
    CK(cudaMemcpyAsync(c->h_offsets, t->offsets, (size_t)(B + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c->h_offsets[0] != 0 || c->h_offsets[B] != t->n_instructions)
        return fail(c, SIMNET_EINVAL, "simulate: offsets[0] must be 0 and offsets[B] = n_instructions");
    int64_t max_len = 0, min_len = INT64_MAX;
    for (int b = 0; b < B; b++) {
        const int64_t n = c->h_offsets[b + 1] - c->h_offsets[b];
        if (n < 0) return fail(c, SIMNET_EINVAL, "simulate: offsets decrease at sub-trace %d", b);
        if (n > 4194303) return fail(c, SIMNET_EINVAL, "simulate: sub-trace %d has %lld instructions (max 4194303)", b, (long long)n);
        max_len = n > max_len ? n : max_len;
        min_len = n < min_len ? n : min_len;
    }
    const uint64_t trace_fp = fnv1a(c->h_offsets, (size_t)(B + 1) * sizeof(int64_t));
    if (resume) {
        if (!c->sim_valid) return fail(c, SIMNET_ESTATE, "simulate: no simulation state to resume");
        if (c->sim_B != B || c->sim_n_inst != t->n_instructions || c->sim_trace_fp != trace_fp)
            return fail(c, SIMNET_ESTATE, "simulate: the trace differs from the one of the held state");
        if (c->sim_weights_fp != weights_fingerprint(c))
            return fail(c, SIMNET_ESTATE, "simulate: the weights differ from the ones of the held state");
    }
    simnet_status st = ensure_workspace(c, B);
    if (st != SIMNET_OK) return st;
    if (c->const_stale && c->cfg.precision != SIMNET_FP32 && (st = refresh_fc1_const(c)) != SIMNET_OK) return st;
    const int64_t done_before = resume ? c->sim_steps : 0;
    const int64_t n_steps = max_steps < 0 ? max_len - done_before : std::min(max_steps, max_len - done_before);

    // per-call arguments -> device (the pinned staging buffer is reused once its last copy is done)
    if (c->args_pending) CK(cudaEventSynchronize(c->args_ev));
    StepArgs &a = *c->h_args;
    a.records = t->records;
    a.offsets = t->offsets;
    a.cycles_out = c->cyc;
    a.lat_log = lat_log;
    a.pre_log = pre_log;
    a.replay = lat_replay;
    a.tick = c->tick;
    a.pos = c->pos;
    a.qstart = c->qstart;
    a.qlen = c->qlen;
    a.evict = c->evict;
    a.ring = c->ring;
    a.active = c->active;
    a.n_active = c->n_active;
    a.status = c->status;
    a.n_sub = B;
    a.window = c->cfg.window;
    a.cap = c->cap;
    a.retire_width = c->cfg.retire_width;
    a.strict = (c->cfg.flags & SIMNET_FLAG_RETIRE_STRICT) ? 1 : 0;
    a.hidden = c->cfg.fc_hidden;
    a.mstart = c->mstart;
    a.mlen = c->mlen;
    a.mring = c->mring;
    a.n_lat = c->n_lat;
    CK(cudaEventRecord(c->ev0, s));
    CK(cudaMemcpyAsync(c->d_args, c->h_args, sizeof(StepArgs), cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->args_ev, s));
    c->args_pending = true;
    if (resume) {
        CK(cudaMemsetAsync(c->status, 0, sizeof(int32_t), s));
    } else {
        launch_init_state(c->d_args, B, s);
        c->sim_valid = true;
        c->sim_B = B;
        c->sim_steps = 0;
        c->sim_max_len = max_len;
        c->sim_n_inst = t->n_instructions;
        c->sim_trace_fp = trace_fp;
        c->sim_weights_fp = weights_fingerprint(c);
    }

    // compaction pays off only when sub-traces finish well apart
    const bool uneven = max_len - min_len > std::max<int64_t>(16, max_len / 8);
    const bool timed = (c->cfg.flags & SIMNET_FLAG_KERNEL_EVENTS) != 0;
    const bool pdl = c->pdl && !timed;
    if ((st = prepare_plans(c, B, pdl)) != SIMNET_OK) return st;
    int64_t launches = 0;
    KTimer kt;
    kt.c = timed ? c : nullptr;
    kt.s = s;
    if (timed) {
        c->ev_used = 0;
        c->kt_valid = false;
    }
    c->phase_valid = false;
    const bool persistent = c->cfg.precision != SIMNET_FP32 && !(c->cfg.flags & SIMNET_FLAG_LAYERWISE);
    const bool fixed = (c->cfg.flags & SIMNET_FLAG_FIXED_PATH) != 0;
    std::string why_not_cluster;
    // the per-layer kernels from the current device state (a gather first: their
    // feature tile is slot-major); CUDA graphs of whole steps unless timed
    auto run_layerwise = [&](int64_t steps) -> simnet_status {
        enqueue_gather(c, B, s, false, timed ? &kt : nullptr);
        launches += 1 + steps * launches_per_step(c);
        if (timed || (c->cfg.flags & SIMNET_FLAG_NO_GRAPH)) {
            for (int64_t i = 0; i < steps; i++) {
                enqueue_step(c, B, s, pdl, timed ? &kt : nullptr);
                if (uneven && (i % kGraphSteps) == kGraphSteps - 1) {
                    enqueue_compact(c, B, s, pdl, timed ? &kt : nullptr);
                    launches += 2;
                }
            }
            if (timed && !kt.ok) return fail(c, SIMNET_ENOMEM, "kernel timing: event pool exhausted");
            c->kt_valid = timed;
        } else {
            simnet_status st2;
            if (c->g_B != B || c->g_compact != (int)uneven || !c->gexec[0])
                if ((st2 = capture_graphs(c, B, uneven)) != SIMNET_OK) return st2;
            const int64_t full = steps / kGraphSteps, rest = steps % kGraphSteps;
            for (int64_t i = 0; i < full; i++) CK(cudaGraphLaunch(c->gexec[0], s));
            for (int64_t i = 0; i < rest; i++) CK(cudaGraphLaunch(c->gexec[1], s));
            if (uneven) launches += 2 * (full + rest);
        }
        c->path = SIMNET_PATH_LAYERWISE;
        return SIMNET_OK;
    };
    auto run_persistent = [&](int64_t steps) -> simnet_status {
        std::string why;
        if (!launch_persistent(c, B, steps, uneven, s, why))
            return fail(c, SIMNET_ECUDA, "persistent kernel: %s", why.c_str());
        launches += 1;
        c->path = SIMNET_PATH_PERSISTENT;
        return SIMNET_OK;
    };
    // Grid-persistent kernel or per-layer kernels for `steps` steps.  The persistent
    // kernel skips the padding rows past the batch's longest queue but pays a grid
    // barrier per phase; per-layer kernels compute every row with cheaper boundaries.
    // Which wins depends on the queue lengths the predictor produces and the batch,
    // so a long untimed call measures both after `warm` steps that let the queues fill:
    // the persistent kernel as two launches (kA and kA + kCmp steps: their difference is
    // its cost per step without the once-per-launch start) and kCmp steps of the
    // per-layer kernels, all from the same state in turn; the path with the smaller
    // estimated cost for the remaining steps runs them.  The pick holds for later calls
    // with the same batch size, compaction and weights.
    auto run_grid_or_layers = [&](int64_t steps, int64_t warm) -> simnet_status {
        constexpr int64_t kA = 16, kCmp = 32, kSpent = 2 * kA + 2 * kCmp;
        simnet_status st2;
        if (timed || fixed || steps < warm + kSpent + 512) return run_persistent(steps);
        const uint64_t wfp = weights_fingerprint(c);
        if (c->pick != SIMNET_PATH_NONE && c->pick_B == B && c->pick_uneven == (int)uneven && c->pick_wfp == wfp)
            return c->pick == SIMNET_PATH_LAYERWISE ? run_layerwise(steps) : run_persistent(steps);
        if (warm > 0 && (st2 = run_persistent(warm)) != SIMNET_OK) return st2;
        if (c->g_B != B || c->g_compact != (int)uneven || !c->gexec[0])   // capture outside the timing
            if ((st2 = capture_graphs(c, B, uneven)) != SIMNET_OK) return st2;
        cudaEvent_t e[4];
        for (auto &x : e) CK(cudaEventCreate(&x));
        CK(cudaEventRecord(e[0], s));
        if ((st2 = run_persistent(kA)) != SIMNET_OK) return st2;
        CK(cudaEventRecord(e[1], s));
        if ((st2 = run_persistent(kA + kCmp)) != SIMNET_OK) return st2;
        CK(cudaEventRecord(e[2], s));
        if ((st2 = run_layerwise(kCmp)) != SIMNET_OK) return st2;
        CK(cudaEventRecord(e[3], s));
        CK(cudaEventSynchronize(e[3]));
        float t_a = 0.f, t_b = 0.f, t_layers = 0.f;
        cudaEventElapsedTime(&t_a, e[0], e[1]);
        cudaEventElapsedTime(&t_b, e[1], e[2]);
        cudaEventElapsedTime(&t_layers, e[2], e[3]);
        for (auto &x : e) cudaEventDestroy(x);
        const int64_t rest = steps - warm - kSpent;
        const double per_grid = std::max(0.0, (double)(t_b - t_a) / kCmp);
        const double start_grid = std::max(0.0, (double)t_a - kA * per_grid);
        const double cost_grid = start_grid + per_grid * (double)rest, cost_layers = (double)t_layers / kCmp * (double)rest;
        // within 3% the persistent kernel stays: its later steps tend to run shorter extents
        c->pick = cost_layers < 0.97 * cost_grid ? SIMNET_PATH_LAYERWISE : SIMNET_PATH_PERSISTENT;
        c->pick_B = B;
        c->pick_uneven = (int)uneven;
        c->pick_wfp = wfp;
        c->pick_ms[0] = (float)(per_grid * kCmp);
        c->pick_ms[1] = t_layers;
        c->pick_steps = (int)kCmp;
        return c->pick == SIMNET_PATH_LAYERWISE ? run_layerwise(rest) : run_persistent(rest);
    };
    launches = resume ? 0 : 1;   // init_state
    if (n_steps <= 0) {
        // nothing to run
    } else if (persistent && !(c->cfg.flags & SIMNET_FLAG_NO_CLUSTER) && cluster_eligible(c, why_not_cluster)) {
        // Clusters own their sub-traces for the whole call: no grid-wide barriers.  Each
        // cluster runs the last-conv positions below its padding extent in passes of a few
        // positions, so when queues stay long the grid-wide or per-layer kernels, which
        // spread the positions over every SM, are faster: the first kProbe steps (queues
        // fill by at most one entry a step) measure the extent over their second half, and
        // the rest of a long call moves on (the state lives in the same device arrays
        // either way).
        constexpr int64_t kProbe = 128;
        c->phase_on = timed;
        if (timed) CK(cudaMemsetAsync(c->phase_ns, 0, 64 * sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(c->phase_ns + 56, 0, 2 * sizeof(unsigned long long), s));
        c->phase_valid = timed;
        std::string why;
        const bool probe = !timed && !fixed && n_steps > 4 * kProbe;
        const int64_t first = probe ? kProbe : n_steps;
        if (!launch_cluster(c, B, first, s, why)) return fail(c, SIMNET_ECUDA, "cluster kernel: %s", why.c_str());
        launches += 1;
        c->path = SIMNET_PATH_CLUSTER;
        if (probe) {
            unsigned long long ps[2] = {0, 0};
            CK(cudaMemcpyAsync(ps, c->phase_ns + 56, sizeof ps, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const int pm = 8 >> (c->cfg.n_conv - 1);   // positions per pass
            const bool long_queues = ps[1] > 0 && (double)ps[0] / (double)ps[1] > 2.0 * pm;
            if (long_queues) {
                c->phase_on = false;
                if ((st = run_grid_or_layers(n_steps - first, 0)) != SIMNET_OK) return st;
            } else {
                if (!launch_cluster(c, B, n_steps - first, s, why))
                    return fail(c, SIMNET_ECUDA, "cluster kernel: %s", why.c_str());
                launches += 1;
            }
        }
    } else if (persistent) {
        // one cooperative kernel runs the steps; its phases are timed by CTA 0 on request
        c->phase_on = timed;
        if (timed) {
            CK(cudaMemsetAsync(c->phase_ns, 0, 64 * sizeof(unsigned long long), s));
            CK(cudaMemsetAsync(c->phase_n, 0, SIMNET_KERNEL_KINDS * sizeof(unsigned long long), s));
        }
        if ((st = run_grid_or_layers(n_steps, 128)) != SIMNET_OK) return st;
        c->phase_valid = timed && c->path == SIMNET_PATH_PERSISTENT;
    } else {
        if ((st = run_layerwise(n_steps)) != SIMNET_OK) return st;
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(cycles_out, c->cyc, (size_t)B * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(c->ev1, s));
    const int64_t done = done_before + std::max<int64_t>(n_steps, 0);
    c->sim_steps = done;
    if (stats) {
        CK(cudaMemsetAsync(c->totals, 0, 2 * sizeof(unsigned long long), s));
        launch_totals(c->d_args, c->totals, B, s);
        CK(cudaMemcpyAsync(c->h_totals, c->totals, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(c->h_status, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        int64_t inst = 0;
        int32_t pending = 0;
        for (int b = 0; b < B; b++) {
            const int64_t n = c->h_offsets[b + 1] - c->h_offsets[b];
            inst += std::max<int64_t>(0, std::min(n, done) - done_before);
            pending += n > done ? 1 : 0;
        }
        stats->total_cycles = (int64_t)c->h_totals[0];
        stats->evictions = (int64_t)c->h_totals[1];
        stats->instructions = inst;
        stats->steps = std::max<int64_t>(n_steps, 0);
        stats->steps_done = done;
        stats->pending = pending;
        stats->kernel_launches = launches;
        stats->ms_total = ms;
        if (*c->h_status != kStatusOk) c->sim_valid = false;
        if (*c->h_status == kStatusTimeout && c->path == SIMNET_PATH_CLUSTER) {
            unsigned long long ti[4] = {0, 0, 0, 0};
            cudaMemcpy(ti, c->phase_ns + 48, sizeof ti, cudaMemcpyDeviceToHost);
            return fail(c, SIMNET_ETIMEOUT,
                        "a device-side wait exceeded its bound (cluster kernel: wait site %llu, CTA %llu, step %lld, "
                        "pass or panel %lld)", ti[0], ti[1], (long long)ti[2], (long long)ti[3]);
        }
        if (*c->h_status == kStatusTimeout) return fail(c, SIMNET_ETIMEOUT, "a device-side wait exceeded its bound");
        if (*c->h_status != kStatusOk) return fail(c, SIMNET_ECUDA, "device status %d", *c->h_status);
    }
    return SIMNET_OK;
}

extern "C" simnet_status simnet_cnn_forward(simnet_ctx *c, const float *x, float *z, int32_t n, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (n < 0 || (n > 0 && (!x || !z))) return fail(c, SIMNET_EINVAL, "cnn_forward: bad arguments");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "cnn_forward: no weights loaded");
    if (n == 0) return SIMNET_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    simnet_status st = ensure_workspace(c, n);
    if (st != SIMNET_OK) return st;
    CK(cudaMemcpyAsync(c->cnt, &n, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // `n` lives on the host stack
    const int64_t rows = (int64_t)n * c->cfg.window;
    switch (c->cfg.precision) {
        case SIMNET_FP32: launch_pack_x<float>(x, (float *)c->X, rows, s); break;
        case SIMNET_BF16: launch_pack_x<__nv_bfloat16>(x, (__nv_bfloat16 *)c->X, rows, s); break;
        default: launch_pack_x<__nv_fp8_e4m3>(x, (__nv_fp8_e4m3 *)c->X, rows, s); break;
    }
    if ((st = prepare_plans(c, n, false)) != SIMNET_OK) return st;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int32_t), s));
    enqueue_cnn(c, c->cnt, n, s, false);
    launch_head_part_z(c->h1, c->n_part, n, c->b2, z, n, c->n_out, s);
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_kernel_times(simnet_ctx *c, float *ms_out, int64_t *launches_out, int32_t n_kinds) {
    if (!c) return SIMNET_EINVAL;
    if (!ms_out || !launches_out || n_kinds < 1 || n_kinds > SIMNET_KERNEL_KINDS)
        return fail(c, SIMNET_EINVAL, "kernel_times: bad arguments");
    if (c->phase_valid && c->path == SIMNET_PATH_CLUSTER)
        return fail(c, SIMNET_ESTATE, "kernel_times: the cluster kernel reports phases through simnet_phase_detail");
    if (c->phase_valid) {  // persistent kernel: per-phase times measured by CTA 0 (globaltimer)
        unsigned long long ns[SIMNET_KERNEL_KINDS], cnt[SIMNET_KERNEL_KINDS];
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(ns, c->phase_ns, sizeof ns, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cnt, c->phase_n, sizeof cnt, cudaMemcpyDeviceToHost));
        for (int k = 0; k < n_kinds; k++) { ms_out[k] = (float)(ns[k] * 1e-6); launches_out[k] = (int64_t)cnt[k]; }
        return SIMNET_OK;
    }
    if (!c->kt_valid) return fail(c, SIMNET_ESTATE, "kernel_times: no timed simulate call");
    CK(cudaDeviceSynchronize());
    for (int k = 0; k < n_kinds; k++) { ms_out[k] = 0.f; launches_out[k] = 0; }
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        const int k = c->ev_kind[i];
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->evpool[i], c->evpool[i + 1]));
        if (k < n_kinds) { ms_out[k] += ms; launches_out[k]++; }
    }
    return SIMNET_OK;
}

extern "C" int32_t simnet_kernel_path(const simnet_ctx *c) { return c ? c->path : -1; }

extern "C" simnet_status simnet_path_choice(const simnet_ctx *c, float *ms_out, int32_t *steps_out) {
    if (!c || !ms_out || !steps_out) return SIMNET_EINVAL;
    ms_out[0] = c->pick_ms[0];
    ms_out[1] = c->pick_ms[1];
    *steps_out = c->pick_steps;
    return SIMNET_OK;
}

extern "C" simnet_status simnet_phase_detail(simnet_ctx *c, uint64_t *out, int32_t n) {
    if (!c) return SIMNET_EINVAL;
    if (!out || n < 1 || n > 48) return fail(c, SIMNET_EINVAL, "phase_detail: bad arguments");
    if (!c->phase_valid) return fail(c, SIMNET_ESTATE, "phase_detail: no timed persistent run");
    CK(cudaDeviceSynchronize());
    const int off = c->path == SIMNET_PATH_CLUSTER ? 0 : 16;
    CK(cudaMemcpy(out, c->phase_ns + off, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return SIMNET_OK;
}

// Autotuner: for a batch of n_sub sub-traces, try every tile width of every
// tensor-core layer (coordinate descent, layer by layer) on a short synthetic
// trace and keep the fastest whole-call device time.
extern "C" simnet_status simnet_autotune(simnet_ctx *c, int32_t n_sub, int32_t steps, int32_t *bn_out,
                                         void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (n_sub < 1 || steps < 1 || steps > 4096) return fail(c, SIMNET_EINVAL, "autotune: bad arguments");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "autotune: no weights loaded");
    if (c->cfg.precision == SIMNET_FP32) return SIMNET_OK;   // the FP32 form has no tile choice
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    // synthetic records (xorshift), equal sub-traces of `steps` instructions
    const int64_t N = (int64_t)n_sub * steps;
    std::vector<uint32_t> rec(N);
    uint64_t st = 0x2545F4914F6CDD1Dull;
    for (int64_t i = 0; i < N; i++) {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        rec[i] = (uint32_t)(st & 0x3ffffffu) & ~(3u << 23) | ((uint32_t)((st >> 40) % 3) << 23);
    }
    std::vector<int64_t> off(n_sub + 1);
    for (int b = 0; b <= n_sub; b++) off[b] = (int64_t)b * steps;
    uint32_t *d_rec = nullptr;
    int64_t *d_off = nullptr, *d_cyc = nullptr;
    auto cleanup = [&]() { cudaFree(d_rec); cudaFree(d_off); cudaFree(d_cyc); };
    if (cudaMalloc(&d_rec, N * 4) != cudaSuccess || cudaMalloc(&d_off, (n_sub + 1) * 8) != cudaSuccess ||
        cudaMalloc(&d_cyc, (size_t)n_sub * 8) != cudaSuccess) {
        cleanup();
        return fail(c, SIMNET_ENOMEM, "autotune: allocation failed");
    }
    cudaMemcpy(d_rec, rec.data(), N * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d_off, off.data(), (n_sub + 1) * 8, cudaMemcpyHostToDevice);
    simnet_trace tr{d_rec, d_off, n_sub, 0, N};
    // one untimed call, then the faster of two timed ones
    auto run = [&](float &ms) -> simnet_status {
        simnet_stats sts;
        simnet_status r = simnet_simulate(c, &tr, d_cyc, nullptr, nullptr, nullptr, &sts, s);
        ms = 1e30f;
        for (int k = 0; r == SIMNET_OK && k < 2; k++) {
            r = simnet_simulate(c, &tr, d_cyc, nullptr, nullptr, nullptr, &sts, s);
            ms = std::min(ms, sts.ms_total);
        }
        return r;
    };
    // coordinate search over one knob at a time, keeping the fastest whole call
    float best = 1e30f;
    auto try_knob = [&](int &knob, std::initializer_list<int> vals, auto ok) -> simnet_status {
        int keep = knob;
        for (int v : vals) {
            if (v == keep || !ok(v)) continue;
            knob = v;
            float ms = 0.f;
            simnet_status r = run(ms);
            if (r != SIMNET_OK) return r;
            if (ms < best) { best = ms; keep = v; }
        }
        knob = keep;
        return SIMNET_OK;
    };
    // start from the built-in rules
    c->tuned_B = -1;
    c->tuned_persist_stages = c->tuned_cluster_size = c->tuned_cluster_stage_bytes = c->tuned_cluster_stages = 0;
    simnet_status r = prepare_plans(c, n_sub, c->pdl);
    if (r != SIMNET_OK) { cleanup(); return r; }
    int cur[kMaxGemm];
    for (int l = 0; l < c->n_layers; l++) cur[l] = c->plan[l].BN;
    c->tuned_B = n_sub;
    for (int l = 0; l < c->n_layers; l++) c->tuned_bn[l] = cur[l];
    if ((r = run(best)) != SIMNET_OK) { cleanup(); return r; }
    c->tuned_path = c->path;
    if (c->path == SIMNET_PATH_CLUSTER) {
        // cluster size, then weight-stage size, then stage count
        const int cs0 = cluster_size_ok(c, 8, n_sub) && c->cfg.fc_hidden / 8 >= 64 ? 8 : 4;
        c->tuned_cluster_size = cs0;
        if ((r = try_knob(c->tuned_cluster_size, {4, 8}, [&](int v) { return cluster_size_ok(c, v, n_sub); })) !=
            SIMNET_OK) { cleanup(); return r; }
        const int CS = c->tuned_cluster_size;
        c->tuned_cluster_stage_bytes = cluster_stage_limit(c, CS, 32768) >= 3 ? 32768 : 16384;
        if ((r = try_knob(c->tuned_cluster_stage_bytes, {16384, 32768},
                          [&](int v) { return cluster_stage_limit(c, CS, v) >= 2; })) != SIMNET_OK) { cleanup(); return r; }
        const int smax = cluster_stage_limit(c, CS, c->tuned_cluster_stage_bytes);
        c->tuned_cluster_stages = smax;
        if ((r = try_knob(c->tuned_cluster_stages, {2, 3, 4, 5, 6, 7, 8}, [&](int v) { return v <= smax; })) !=
            SIMNET_OK) { cleanup(); return r; }
    } else {
        // tile width of every tensor-core GEMM (the persistent kernel's phases and the
        // per-layer kernels take the same plans), then the persistent kernel's stages
        for (int l = 0; l < c->n_layers; l++) {
            const int N = c->layer[l].N;
            if ((r = try_knob(c->tuned_bn[l], {64, 128, 256}, [&](int v) { return N % v == 0; })) != SIMNET_OK) {
                cleanup();
                return r;
            }
            cur[l] = c->tuned_bn[l];
        }
        if (c->path == SIMNET_PATH_PERSISTENT) {
            c->tuned_persist_stages = 6;
            if ((r = try_knob(c->tuned_persist_stages, {2, 3, 4, 5}, [](int) { return true; })) != SIMNET_OK) {
                cleanup();
                return r;
            }
        }
    }
    cleanup();
    if (bn_out)
        for (int l = 0; l < c->n_layers; l++) bn_out[l] = c->tuned_bn[l];
    return SIMNET_OK;
}

extern "C" simnet_status simnet_autotune_plan(const simnet_ctx *c, int32_t *out, int32_t n) {
    if (!c || !out || n < 6) return SIMNET_EINVAL;
    const int32_t head[6] = {c->tuned_B, c->tuned_path, c->tuned_cluster_size, c->tuned_cluster_stage_bytes,
                             c->tuned_cluster_stages, c->tuned_persist_stages};
    for (int i = 0; i < n; i++) out[i] = i < 6 ? head[i] : (i - 6 < c->n_layers ? c->tuned_bn[i - 6] : 0);
    return SIMNET_OK;
}
