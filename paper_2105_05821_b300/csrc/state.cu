// state.cu -- checkpoint / resume: export and import of the simulation state
// (per-sub-trace curTick, position, processor-queue ring and counters of the
// lock-step loop, Sec. 3.2-3.3) and of the training state (FP32 master
// weights, Adam moments and step count, Sec. 2.4).
//
// Format: a fixed header followed by the raw arrays, little-endian, in the
// order listed below.  The header carries the config fields that shape the
// arrays; a state loads only into a context whose fields match.
#include <cstring>
#include <vector>

#include "ctx.cuh"

namespace {

constexpr char kMagic[8] = {'S', 'I', 'M', 'N', 'E', 'T', 'S', '1'};
constexpr int32_t kVersion = 2;   // 2: ring entries carry S and a 22-bit fetch tick

struct StateHeader {
    char magic[8];
    int32_t version, kind;
    int32_t window, n_conv, conv_channels, fc_hidden;
    int32_t retire_width, strict, precision, n_sub;
    int32_t cap, head;   // head: bit 0 hybrid FC2, bit 1 store latency + memory write queue
    int64_t steps_done, max_len, n_instructions;
    uint64_t trace_fp, weights_fp;
    int64_t payload_bytes;
};
static_assert(sizeof(StateHeader) == 104, "state header layout");

// SIM payload: tick, pos, qstart, qlen, evict, active (int32 [B] each),
// n_active (int64), finished cycles (int64 [B]), ring (uint64 [B][cap]); with
// the memory write queue then mstart, mlen (int32 [B]) and its ring (uint64 [B][cap]).
size_t sim_payload(int B, int cap, bool sq) {
    return (size_t)B * 6 * 4 + 8 + (size_t)B * 8 + (size_t)B * cap * 8 + (sq ? (size_t)B * 8 + (size_t)B * cap * 8 : 0);
}

// TRAIN payload: canonical FP32 weights [n_weights], step (int64), then per
// GEMM layer l the Adam moments m, v of its weights (FP32 [N][K], GEMM
// layout) and of its bias ([N]); then m, v of FC2's weights [n_out*H] and bias [n_out].
size_t train_payload(const simnet_ctx *c) {
    size_t n = (size_t)c->n_weights * 4 + 8;
    for (int l = 0; l < c->n_layers; l++) n += 2 * ((size_t)c->layer[l].N * c->layer[l].K + c->layer[l].N) * 4;
    return n + 2 * ((size_t)c->n_out * c->cfg.fc_hidden + c->n_out) * 4;
}

void fill_header(const simnet_ctx *c, int kind, StateHeader &h) {
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.kind = kind;
    h.window = c->cfg.window;
    h.n_conv = c->cfg.n_conv;
    h.conv_channels = c->cfg.conv_channels;
    h.fc_hidden = c->cfg.fc_hidden;
    h.retire_width = c->cfg.retire_width;
    h.strict = (c->cfg.flags & SIMNET_FLAG_RETIRE_STRICT) ? 1 : 0;
    h.precision = c->cfg.precision;
    h.cap = c->cap;
    h.head = (c->hybrid ? 1 : 0) | (c->store_queue ? 2 : 0);
}

}  // namespace

extern "C" simnet_status simnet_state_save(simnet_ctx *c, int32_t kind, void *host_buf, size_t *bytes,
                                           void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!bytes || (kind != SIMNET_STATE_SIM && kind != SIMNET_STATE_TRAIN))
        return fail(c, SIMNET_EINVAL, "state_save: bad kind or NULL size");
    if (kind == SIMNET_STATE_SIM && !c->sim_valid) return fail(c, SIMNET_ESTATE, "state_save: no simulation state");
    if (kind == SIMNET_STATE_TRAIN && !c->has_weights) return fail(c, SIMNET_ESTATE, "state_save: no weights loaded");
    const size_t payload = kind == SIMNET_STATE_SIM ? sim_payload(c->sim_B, c->cap, c->store_queue) : train_payload(c);
    const size_t need = sizeof(StateHeader) + payload;
    if (!host_buf) {
        *bytes = need;
        return SIMNET_OK;
    }
    if (*bytes < need) return fail(c, SIMNET_EINVAL, "state_save: buffer of %zu bytes, need %zu", *bytes, need);
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    StateHeader h;
    fill_header(c, kind, h);
    h.payload_bytes = (int64_t)payload;
    uint8_t *out = (uint8_t *)host_buf;
    size_t off = sizeof h;
    auto get = [&](const void *dev, size_t n) -> cudaError_t {
        cudaError_t e = cudaMemcpy(out + off, dev, n, cudaMemcpyDeviceToHost);
        off += n;
        return e;
    };
    if (kind == SIMNET_STATE_SIM) {
        const int B = c->sim_B;
        h.n_sub = B;
        h.steps_done = c->sim_steps;
        h.max_len = c->sim_max_len;
        h.n_instructions = c->sim_n_inst;
        h.trace_fp = c->sim_trace_fp;
        h.weights_fp = c->sim_weights_fp;
        const int32_t *arr[] = {c->tick, c->pos, c->qstart, c->qlen, c->evict, c->active};
        for (const int32_t *a : arr) CK(get(a, (size_t)B * 4));
        int32_t na = 0;
        CK(cudaMemcpy(&na, c->n_active, 4, cudaMemcpyDeviceToHost));
        const int64_t na64 = na;
        memcpy(out + off, &na64, 8);
        off += 8;
        CK(get(c->cyc, (size_t)B * 8));
        CK(get(c->ring, (size_t)B * c->cap * 8));
        if (c->store_queue) {
            CK(get(c->mstart, (size_t)B * 4));
            CK(get(c->mlen, (size_t)B * 4));
            CK(get(c->mring, (size_t)B * c->cap * 8));
        }
    } else {
        h.weights_fp = weights_fingerprint(c);
        simnet_status st = simnet_get_weights(c, (float *)(out + off));
        if (st != SIMNET_OK) return st;
        off += (size_t)c->n_weights * 4;
        const TrainState &t = c->tr;
        const int64_t step = t.ready ? t.step : 0;
        memcpy(out + off, &step, 8);
        off += 8;
        auto put = [&](const float *dev, size_t n) -> cudaError_t {
            if (!t.ready) {   // no optimiser yet: zero moments
                memset(out + off, 0, n * 4);
                off += n * 4;
                return cudaSuccess;
            }
            return get(dev, n * 4);
        };
        for (int l = 0; l < c->n_layers; l++) {
            const size_t wn = (size_t)c->layer[l].N * c->layer[l].K, nb = c->layer[l].N;
            CK(put(t.mW[l], wn));
            CK(put(t.vW[l], wn));
            CK(put(t.mb[l], nb));
            CK(put(t.vb[l], nb));
        }
        const size_t h2 = (size_t)c->n_out * c->cfg.fc_hidden;
        CK(put(t.mw2, h2));
        CK(put(t.vw2, h2));
        CK(put(t.mb2, (size_t)c->n_out));
        CK(put(t.vb2, (size_t)c->n_out));
    }
    memcpy(out, &h, sizeof h);
    *bytes = off;
    return SIMNET_OK;
}

extern "C" simnet_status simnet_state_load(simnet_ctx *c, int32_t kind, const void *host_buf, size_t bytes,
                                           void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!host_buf || (kind != SIMNET_STATE_SIM && kind != SIMNET_STATE_TRAIN))
        return fail(c, SIMNET_EINVAL, "state_load: bad kind or NULL buffer");
    if (bytes < sizeof(StateHeader)) return fail(c, SIMNET_EINVAL, "state_load: %zu bytes is shorter than a header", bytes);
    StateHeader h;
    memcpy(&h, host_buf, sizeof h);
    if (memcmp(h.magic, kMagic, 8) != 0) return fail(c, SIMNET_EINVAL, "state_load: not a state (bad magic)");
    if (h.version != kVersion) return fail(c, SIMNET_EINVAL, "state_load: format version %d, expected %d", h.version, kVersion);
    if (h.kind != kind) return fail(c, SIMNET_EINVAL, "state_load: the buffer holds state kind %d", h.kind);
    StateHeader mine;
    fill_header(c, kind, mine);
    if (h.window != mine.window || h.n_conv != mine.n_conv || h.conv_channels != mine.conv_channels ||
        h.fc_hidden != mine.fc_hidden || h.head != mine.head)
        return fail(c, SIMNET_EINVAL, "state_load: state of another CNN shape (W=%d, %d x conv%d, FC%d, %s head%s)",
                    h.window, h.n_conv, h.conv_channels, h.fc_hidden, (h.head & 1) ? "hybrid" : "regression",
                    (h.head & 2) ? ", write queue" : "");
    const uint8_t *in = (const uint8_t *)host_buf;
    size_t off = sizeof h;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    auto put = [&](void *dev, size_t n) -> cudaError_t {
        cudaError_t e = cudaMemcpy(dev, in + off, n, cudaMemcpyHostToDevice);
        off += n;
        return e;
    };
    if (kind == SIMNET_STATE_SIM) {
        if (h.retire_width != mine.retire_width || h.strict != mine.strict || h.cap != mine.cap)
            return fail(c, SIMNET_EINVAL, "state_load: state of another retire width, retire rule or queue capacity");
        const int B = h.n_sub;
        const size_t pl = sim_payload(B, h.cap, c->store_queue);
        if (B < 1 || h.steps_done < 0 || h.steps_done > h.max_len || h.payload_bytes != (int64_t)pl ||
            bytes != sizeof h + pl)
            return fail(c, SIMNET_EINVAL, "state_load: inconsistent simulation state header or size");
        simnet_status st = ensure_workspace(c, B);
        if (st != SIMNET_OK) return st;
        int32_t *arr[] = {c->tick, c->pos, c->qstart, c->qlen, c->evict, c->active};
        for (int32_t *a : arr) CK(put(a, (size_t)B * 4));
        int64_t na64 = 0;
        memcpy(&na64, in + off, 8);
        off += 8;
        if (na64 < 0 || na64 > B) return fail(c, SIMNET_EINVAL, "state_load: active count %lld of %d", (long long)na64, B);
        const int32_t na = (int32_t)na64;
        CK(cudaMemcpy(c->n_active, &na, 4, cudaMemcpyHostToDevice));
        CK(put(c->cyc, (size_t)B * 8));
        CK(put(c->ring, (size_t)B * c->cap * 8));
        if (c->store_queue) {
            CK(put(c->mstart, (size_t)B * 4));
            CK(put(c->mlen, (size_t)B * 4));
            CK(put(c->mring, (size_t)B * c->cap * 8));
        }
        c->sim_valid = true;
        c->sim_B = B;
        c->sim_steps = h.steps_done;
        c->sim_max_len = h.max_len;
        c->sim_n_inst = h.n_instructions;
        c->sim_trace_fp = h.trace_fp;
        c->sim_weights_fp = h.weights_fp;
        return SIMNET_OK;
    }
    if (h.payload_bytes != (int64_t)train_payload(c) || bytes != sizeof h + train_payload(c))
        return fail(c, SIMNET_EINVAL, "state_load: inconsistent training state size");
    std::vector<float> blob((size_t)c->n_weights);
    memcpy(blob.data(), in + off, blob.size() * 4);
    off += blob.size() * 4;
    simnet_status st = simnet_load_weights(c, blob.data(), c->n_weights);
    if (st != SIMNET_OK) return st;
    int64_t step = 0;
    memcpy(&step, in + off, 8);
    off += 8;
    if ((c->cfg.precision != SIMNET_FP32 && c->cfg.precision != SIMNET_BF16) || c->residual)
        return SIMNET_OK;  // FP8 and residual contexts do not train: weights only
    if ((st = ensure_train(c, 0)) != SIMNET_OK) return st;
    TrainState &t = c->tr;
    for (int l = 0; l < c->n_layers; l++) {
        const size_t wn = (size_t)c->layer[l].N * c->layer[l].K, nb = c->layer[l].N;
        CK(put(t.mW[l], wn * 4));
        CK(put(t.vW[l], wn * 4));
        CK(put(t.mb[l], nb * 4));
        CK(put(t.vb[l], nb * 4));
    }
    const size_t h2 = (size_t)c->n_out * c->cfg.fc_hidden;
    CK(put(t.mw2, h2 * 4));
    CK(put(t.vw2, h2 * 4));
    CK(put(t.mb2, (size_t)c->n_out * 4));
    CK(put(t.vb2, (size_t)c->n_out * 4));
    t.step = step;
    return SIMNET_OK;
}
