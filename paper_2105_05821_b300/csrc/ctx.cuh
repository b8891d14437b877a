// ctx.cuh -- the library context (simnet_ctx) shared by the host-side files.
#pragma once
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"
#include "train_tc.cuh"

using namespace simnet;

// Training state: Adam moments, gradients and the saved activations of the last
// training forward (the FP32 master weights are the context's W32/bias/w2/b2).
struct TrainState {
    bool ready = false;
    int n_cap = 0;                     // windows the buffers hold
    int64_t step = 0;                  // Adam step counter
    float *gW[kMaxGemm] = {}, *gb[kMaxGemm] = {};    // gradients
    float *mW[kMaxGemm] = {}, *vW[kMaxGemm] = {};    // Adam moments (weights)
    float *mb[kMaxGemm] = {}, *vb[kMaxGemm] = {};    // Adam moments (biases)
    float *gw2 = nullptr, *gb2 = nullptr;
    float *mw2 = nullptr, *vw2 = nullptr, *mb2 = nullptr, *vb2 = nullptr;
    float *X = nullptr;                // packed input [n][W][64]
    float *Y[kMaxGemm] = {};           // outputs of every layer (post-ReLU); Y[L] = FC1 [n][H]
    float *dA = nullptr, *dB = nullptr;  // gradient ping-pong buffers (largest activation)
    float *z = nullptr, *dz = nullptr; // [n][n_out]
    double *loss = nullptr;            // device scalar
    int n_last = 0;                    // windows of the last forward
    // BF16 contexts train on the tensor cores: BF16 operands and saved activations
    __nv_bfloat16 *Xb = nullptr;           // packed input [n][W][64]
    __nv_bfloat16 *Yb[kMaxGemm] = {};      // conv outputs [n * m_mult][N] (post-ReLU)
    __nv_bfloat16 *dHb = nullptr;          // dLoss / d(FC1 output) [n][H] (ReLU applied)
    __nv_bfloat16 *dYb[2] = {};            // conv-output gradients, ping-pong (largest activation)
    TgPlan fwd[kMaxGemm], wgrad[kMaxGemm], dgrad[kMaxGemm];
    int plan_n = -1;                       // windows the plans were built for
    float *colpart = nullptr;              // per-block column sums of the bias gradients
    float *wpart = nullptr;                // split partial tiles of the weight gradients
    size_t wpart_cap = 0;                  // floats
};

struct simnet_ctx {
    simnet_config cfg{};
    int cap = 0, rows_n = 0, fc1_in = 0, n_layers = 0;
    int n_lat = 2;   // latencies per instruction: fetch, execution (and store, with the write queue)
    bool hybrid = false, store_queue = false;
    int n_out = 2;   // FC2 outputs: n_lat (regression head) or 11 * n_lat (hybrid head)
    int64_t n_weights = 0;
    std::string err;
    bool has_weights = false;
    int device = 0;

    // weights in GEMM layout ([N][K], layer precision) + FP32 biases; FC2 in FP32
    void *Wl[kMaxGemm] = {};
    float *bias[kMaxGemm] = {};
    float *wscale[kMaxGemm] = {};  // FP8: per-output-channel dequant scale
    float *oscale[kMaxGemm] = {};  // FP8: per-output-channel requant multiplier (1/next act scale)
    float *W32[kMaxGemm] = {};     // FP32 GEMM-layout weights (aliases Wl for FP32 contexts)
    float *w2 = nullptr, *b2 = nullptr;
    GemmLayer layer[kMaxGemm];
    TcPlan plan[kMaxGemm];
    // residual blocks (SIMNET_FLAG_RESIDUAL): GEMMs 3b, 3b+1, 3b+2 are block b's
    // conv, projection shortcut and pointwise conv (+ shortcut); the canonical
    // blob is kept on the host (these contexts do not train on the device)
    bool residual = false;
    int n_blocks = 0;
    std::vector<float> blob_host;

    // workspace, sized for ws_B sub-traces
    int ws_B = 0;
    void *X = nullptr, *act[2] = {nullptr, nullptr};
    void *tmpA = nullptr, *tmpS = nullptr;   // residual blocks: branch and shortcut [B][W/2][C]
    float *h1 = nullptr;  // FC2 partial sums [n_part][B][n_out] float
    int n_part = 0;
    bool pdl = true;
    int32_t *tick = nullptr, *pos = nullptr, *qstart = nullptr, *qlen = nullptr, *evict = nullptr;
    int32_t *active = nullptr, *n_active = nullptr, *status = nullptr, *cnt = nullptr;
    uint64_t *ring = nullptr;
    int32_t *mstart = nullptr, *mlen = nullptr;   // memory write queue (store-queue contexts)
    uint64_t *mring = nullptr;
    unsigned long long *totals = nullptr;
    StepArgs *d_args = nullptr, *h_args = nullptr;
    int64_t *h_offsets = nullptr;
    size_t h_offsets_cap = 0;
    unsigned long long *h_totals = nullptr;
    int32_t *h_status = nullptr;
    cudaEvent_t args_ev = nullptr, ev0 = nullptr, ev1 = nullptr;
    bool args_pending = false;
    cudaStream_t cap_stream = nullptr;

    // captured step graphs: [0] = kGraphSteps steps, [1] = one step
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int g_B = -1, g_compact = -1;

    // per-kernel CUDA-event timing (SIMNET_FLAG_KERNEL_EVENTS)
    std::vector<cudaEvent_t> evpool;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    bool kt_valid = false;

    TrainState tr;

    // persistent kernel: grid barrier counter, abort flag, per-phase times (CTA 0)
    unsigned *bar = nullptr;
    int *bar_abort = nullptr;
    unsigned long long *phase_ns = nullptr, *phase_n = nullptr;
    bool phase_on = false, phase_valid = false;

    // padding-extent path of the persistent kernel: FC1 contribution of the
    // constant rows past the extent, S[e][n] for e = 0..rows_n ([rows_n+1][H]),
    // and the batch extent per step parity
    float *fc1_const = nullptr;
    int *ext = nullptr;
    // per-layer extent: each conv-stack layer's constant output row in storage
    // units ([n_layers - 1][C]) and the layers' private output tiles (pair-major,
    // sized for pbuf_B sub-traces) that keep those constants past the extent
    float *layer_const = nullptr;
    void *pbuf[kMaxGemm] = {};
    int pbuf_B = 0;

    // autotuned launch shapes, for batches of tuned_B sub-traces (0 = the built-in
    // rule): tile widths of the tensor-core GEMMs (per-layer and persistent kernels),
    // the persistent kernel's pipeline stages, the cluster kernel's cluster size,
    // weight-stage bytes and stage count
    int tuned_B = -1;
    int tuned_bn[kMaxGemm] = {};
    int tuned_persist_stages = 0;
    int tuned_cluster_size = 0, tuned_cluster_stage_bytes = 0, tuned_cluster_stages = 0;
    int tuned_path = SIMNET_PATH_NONE;   // the path the tuning ran on

    // resumable simulation state: the workspace arrays tick/pos/qstart/qlen/
    // evict/ring/active/n_active plus the finished cycle counts `cyc`
    int64_t *cyc = nullptr;   // [ws_B]
    bool sim_valid = false;
    int sim_B = 0;
    int64_t sim_steps = 0, sim_max_len = 0, sim_n_inst = 0;
    uint64_t sim_trace_fp = 0, sim_weights_fp = 0;

    // fingerprint of the FP32 weights (recomputed lazily after on-device updates)
    uint64_t weights_fp = 0;
    bool weights_fp_dirty = false;
    // the padding-constant table fc1_const no longer matches the weights (set by
    // on-device weight updates; rebuilt before the next persistent run)
    bool const_stale = false;
    int path = SIMNET_PATH_NONE;   // kernel path of the last simulate call
    // the grid-wide path picked by the last timed comparison (SIMNET_PATH_PERSISTENT or
    // SIMNET_PATH_LAYERWISE) and what it was measured for: batch size, compaction, weights
    int pick = SIMNET_PATH_NONE, pick_B = -1, pick_uneven = -1;
    uint64_t pick_wfp = 0;
    float pick_ms[2] = {0.f, 0.f};   // the comparison's persistent / per-layer times
    int pick_steps = 0;
};

namespace simnet {
bool launch_persistent(simnet_ctx *c, int B, int64_t n_steps, bool uneven, cudaStream_t s, std::string &why);
// Cluster kernel (cluster.cu): every simulate step without grid-wide barriers,
// for the shapes cluster_eligible accepts.
bool cluster_eligible(const simnet_ctx *c, std::string &why);
bool launch_cluster(simnet_ctx *c, int B, int64_t n_steps, cudaStream_t s, std::string &why);
// Autotuner support: whether clusters of CS CTAs can run a batch of B, and the most
// weight stages of stage_bytes that fit with them (0 if none).
bool cluster_size_ok(const simnet_ctx *c, int CS, int B);
int cluster_stage_limit(const simnet_ctx *c, int CS, int stage_bytes);
}

// Training buffers for n windows (and the optimiser state, once); train.cu.
simnet_status ensure_train(simnet_ctx *c, int n);
// Simulation workspaces for B sub-traces (reallocating drops a held state).
simnet_status ensure_workspace(simnet_ctx *c, int B);
// Fingerprint of the FP32 weights in canonical order (0 if they cannot be read).
uint64_t weights_fingerprint(simnet_ctx *c);
// Tabulate fc1_const from FP32 biases and the weights as the kernels use them
// (GEMM layout, dequantised); osc = FP8 requant multipliers (empty otherwise).
simnet_status build_fc1_const(simnet_ctx *c, const std::vector<std::vector<float>> &Bg,
                              const std::vector<std::vector<float>> &Wdeq,
                              const std::vector<std::vector<float>> &osc);
// Rebuild fc1_const from the FP32 master weights on the device (BF16 contexts
// after on-device updates).
simnet_status refresh_fc1_const(simnet_ctx *c);
// 64-bit FNV-1a of a byte range, continuing from h.
inline uint64_t fnv1a(const void *p, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    const uint8_t *b = (const uint8_t *)p;
    for (size_t i = 0; i < n; i++) { h ^= b[i]; h *= 0x100000001b3ull; }
    return h;
}

// Records an event pair around each kernel when timing is on.
struct KTimer {
    simnet_ctx *c = nullptr;
    cudaStream_t s = nullptr;
    bool ok = true;
    void begin(int kind) {
        if (!c) return;
        if (c->ev_used + 2 > c->evpool.size()) {
            for (int i = 0; i < 256; i++) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) { ok = false; return; }
                c->evpool.push_back(e);
            }
            c->ev_kind.resize(c->evpool.size());
        }
        c->ev_kind[c->ev_used] = kind;
        cudaEventRecord(c->evpool[c->ev_used++], s);
    }
    void end() {
        if (!c || !ok) return;
        cudaEventRecord(c->evpool[c->ev_used++], s);
    }
};


static inline simnet_status fail(simnet_ctx *c, simnet_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(c, e_ == cudaErrorMemoryAllocation ? SIMNET_ENOMEM : SIMNET_ECUDA,        \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

