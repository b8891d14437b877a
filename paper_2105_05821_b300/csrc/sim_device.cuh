// sim_device.cuh -- device-side pieces of a simulation step shared by the
// per-step kernels and the persistent kernel: context gather (Sec. 2.2), the
// latency head and processor-queue / curTick update (Sec. 3.2), the drain of
// Eq. 1 (Sec. 3.1) and active-set compaction (Sec. 3.3).
#pragma once
#include "common.cuh"

namespace simnet {

// ------------------------------------------------------------------ vector stores per precision
template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int N = 4; };
template <> struct Vec<__nv_bfloat16> { static constexpr int N = 8; };
template <> struct Vec<__nv_fp8_e4m3> { static constexpr int N = 16; };

template <typename T> __device__ __forceinline__ void store16(T *dst, const float *v);

template <> __device__ __forceinline__ void store16<float>(float *dst, const float *v) {
    *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void store16<__nv_bfloat16>(__nv_bfloat16 *dst, const float *v) {
    uint4 u;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
    u.x = *reinterpret_cast<uint32_t *>(&p0);
    u.y = *reinterpret_cast<uint32_t *>(&p1);
    u.z = *reinterpret_cast<uint32_t *>(&p2);
    u.w = *reinterpret_cast<uint32_t *>(&p3);
    *reinterpret_cast<uint4 *>(dst) = u;
}
template <> __device__ __forceinline__ void store16<__nv_fp8_e4m3>(__nv_fp8_e4m3 *dst, const float *v) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * q], v[4 * q + 1]), __NV_SATFINITE, __NV_E4M3);
        uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * q + 2], v[4 * q + 3]), __NV_SATFINITE, __NV_E4M3);
        w[q] = (lo & 0xffffu) | (hi << 16);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// ------------------------------------------------------------------ whole-row feature writer
// Channels 32..63 of a row (the part after the opcode one-hot), as floats.
__device__ __forceinline__ void row_tail(uint32_t rec, uint32_t cur, bool ctx, int32_t res, uint32_t e,
                                         uint32_t s, float (&t)[32]) {
#pragma unroll
    for (int j = 0; j < 32; j++) t[j] = 0.f;
    const uint32_t dst = (rec >> 15) & 31u, lvl = (rec >> 23) & 3u;
    t[0] = (float)((rec >> 5) & 31u) * 0.03125f;
    t[1] = (float)((rec >> 10) & 31u) * 0.03125f;
    t[2] = (float)dst * 0.03125f;
    t[3] = (float)((rec >> 20) & 1u);
    t[4] = (float)((rec >> 21) & 1u);
    t[5] = (float)((rec >> 22) & 1u);
    t[6] = lvl == 0u ? 1.f : 0.f;
    t[7] = lvl == 1u ? 1.f : 0.f;
    t[8] = lvl == 2u ? 1.f : 0.f;
    t[9] = (float)((rec >> 25) & 1u);
    if (ctx) {
        t[10] = (float)min(res, 4095) * 0.015625f;
        t[11] = (float)e * 0.015625f;
        t[12] = rec_is_store(rec) ? (float)s * 0.015625f : 0.f;
        t[13] = dst == ((cur >> 5) & 31u) ? 1.f : 0.f;
        t[14] = dst == ((cur >> 10) & 31u) ? 1.f : 0.f;
        t[15] = dst == ((cur >> 15) & 31u) ? 1.f : 0.f;
        const bool m0 = (rec >> 20) & 3u, m1 = (cur >> 20) & 3u;
        t[16] = (m0 && m1 && lvl == ((cur >> 23) & 3u)) ? 1.f : 0.f;
    }
}

// Write one whole 64-channel row (same values as `feature` channel by channel).
template <typename T> __device__ __forceinline__ void write_row(T *dst, uint32_t rec, uint32_t cur, bool ctx,
                                                               int32_t res, uint32_t e, uint32_t s);

// A BF16 row as its eight 16-byte chunks (channels 8j .. 8j+7 in chunk j).
__device__ __forceinline__ void row_chunks_bf16(uint32_t rec, uint32_t cur, bool ctx, int32_t res, uint32_t e,
                                                uint32_t s, uint4 (&o)[8]) {
    const uint32_t op = rec & 31u;
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; i++) w[i] = (op >> 1) == (uint32_t)i ? ((op & 1u) ? 0x3F800000u : 0x00003F80u) : 0u;
#pragma unroll
    for (int i = 0; i < 4; i++) o[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    float t[32];
    row_tail(rec, cur, ctx, res, e, s, t);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        __nv_bfloat162 b = __floats2bfloat162_rn(t[2 * i], t[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&b);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) o[4 + i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
}

template <> __device__ __forceinline__ void write_row<__nv_bfloat16>(__nv_bfloat16 *dst, uint32_t rec, uint32_t cur,
                                                                     bool ctx, int32_t res, uint32_t e, uint32_t s) {
    uint4 o[8];
    row_chunks_bf16(rec, cur, ctx, res, e, s, o);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 8; i++) d4[i] = o[i];
}

// An FP8 e4m3 row as its four 16-byte chunks (channels 16j .. 16j+15 in chunk j).
__device__ __forceinline__ void row_chunks_fp8(uint32_t rec, uint32_t cur, bool ctx, int32_t res, uint32_t e,
                                               uint32_t s, uint4 (&o)[4]) {
    const uint32_t op = rec & 31u;
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; i++) w[i] = (op >> 2) == (uint32_t)i ? (0x38u << (8 * (op & 3u))) : 0u;  // e4m3 1.0
    o[0] = make_uint4(w[0], w[1], w[2], w[3]);
    o[1] = make_uint4(w[4], w[5], w[6], w[7]);
    float t[32];
    row_tail(rec, cur, ctx, res, e, s, t);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(t[4 * i], t[4 * i + 1]), __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(t[4 * i + 2], t[4 * i + 3]), __NV_SATFINITE, __NV_E4M3);
        w[i] = (lo & 0xffffu) | (hi << 16);
    }
    o[2] = make_uint4(w[0], w[1], w[2], w[3]);
    o[3] = make_uint4(w[4], w[5], w[6], w[7]);
}

template <> __device__ __forceinline__ void write_row<__nv_fp8_e4m3>(__nv_fp8_e4m3 *dst, uint32_t rec, uint32_t cur,
                                                                     bool ctx, int32_t res, uint32_t e, uint32_t s) {
    uint4 o[4];
    row_chunks_fp8(rec, cur, ctx, res, e, s, o);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 4; i++) d4[i] = o[i];
}

template <> __device__ __forceinline__ void write_row<float>(float *dst, uint32_t rec, uint32_t cur, bool ctx,
                                                             int32_t res, uint32_t e, uint32_t s) {
    const uint32_t op = rec & 31u;
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] = op == (uint32_t)(4 * i + j) ? 1.f : 0.f;
        d4[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
    float t[32];
    row_tail(rec, cur, ctx, res, e, s, t);
#pragma unroll
    for (int i = 0; i < 8; i++) d4[8 + i] = make_float4(t[4 * i], t[4 * i + 1], t[4 * i + 2], t[4 * i + 3]);
}

__device__ __forceinline__ void zero_row_bytes(void *dst, int bytes) {
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int i = 0; i < bytes / 16; i++) d4[i] = make_uint4(0, 0, 0, 0);
}

// ------------------------------------------------------------------ head + queue update (Sec. 3.2)
__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// clamp to [0, 255], round half to even; NaN -> 255
__device__ __forceinline__ uint32_t to_cycles(float y) {
    if (isnan(y)) return 255u;
    y = fminf(fmaxf(y, 0.f), 255.f);
    return (uint32_t)__float2int_rn(y);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FC2 outputs per window: a regression head has one per latency (2, or 3 with
// the store latency); a hybrid head has eleven per latency (22 or 33).
template <int NO> constexpr bool out_hybrid() { return NO % 11 == 0; }
template <int NO> constexpr int out_lat() { return out_hybrid<NO>() ? NO / 11 : NO; }

// Latency T (0 fetch, 1 execution, 2 store) from the FC2 outputs z[0..NO) (bias
// included); `pre` receives the softplus value before clamping and rounding.
// Regression head: round(clamp(softplus(z[T]))).  Hybrid head (Sec. 2.3): the
// class k with the largest of the ten logits z[11T..11T+9], compared in FP32
// with the lowest index winning ties; classes 0..8 are the latency itself,
// class 9 ("more than 8") takes the regression output z[11T+10].
template <int NO, int T>
__device__ __forceinline__ uint32_t head_latency(const float (&z)[NO], float &pre) {
    if constexpr (!out_hybrid<NO>()) {
        pre = softplus_f(z[T]);
        return to_cycles(pre);
    } else {
        float lg[11];
#pragma unroll
        for (int j = 0; j < 11; j++) lg[j] = z[11 * T + j];
        float best = lg[0];
        int k = 0;
#pragma unroll
        for (int j = 1; j < 10; j++)
            if (lg[j] > best) { best = lg[j]; k = j; }
        pre = softplus_f(lg[10]);
        return k <= 8 ? (uint32_t)k : to_cycles(pre);
    }
}

// FC2 outputs of one slot, in every lane of the warp: z[o] = b2[o] + the sum
// over the P partials part[(i * part_stride + slot) * NO + o].
template <int NO>
__device__ __forceinline__ void head_sum_warp(const float *__restrict__ part, int P, int part_stride, int slot,
                                              const float *__restrict__ b2, int lane, float (&z)[NO]) {
    if constexpr (NO == 2) {
        float zf = 0.f, ze = 0.f;
        for (int i = lane; i < P; i += 32) {
            const float2 v = reinterpret_cast<const float2 *>(part)[(size_t)i * part_stride + slot];
            zf += v.x;
            ze += v.y;
        }
        z[0] = warp_sum(zf) + b2[0];
        z[1] = warp_sum(ze) + b2[1];
    } else {
        // lane l adds outputs l and l + 32 over the partials, then every lane gets all NO
        constexpr int NA = (NO + 31) / 32;
        float acc[NA];
#pragma unroll
        for (int a = 0; a < NA; a++) {
            const int o = a * 32 + lane;
            acc[a] = 0.f;
            if (o < NO) {
                acc[a] = b2[o];
                for (int i = 0; i < P; i++) acc[a] += part[((size_t)i * part_stride + slot) * NO + o];
            }
        }
#pragma unroll
        for (int o = 0; o < NO; o++) z[o] = __shfl_sync(0xffffffffu, acc[o / 32], o % 32);
    }
}

// Length of the run of ready entries from the oldest, at most `lim`; in-order
// retire means the first not-ready entry stops it.  Ready: residence reaches E
// (processor queue) or, with STORE_LAT, S (memory write queue).  Whole warp
// participates.
template <bool STORE_LAT = false>
__device__ __forceinline__ int retire_run(const uint64_t *__restrict__ ring, int cap, int qs, int lim,
                                          int32_t tick, int strict, int lane) {
    int k = 0;
    while (k < lim) {
        const int i = k + lane;
        bool rd = false;
        if (i < lim) {
            int idx = qs + i;
            if (idx >= cap) idx -= cap;
            const uint64_t v = ring[idx];
            const int32_t res = entry_res(v, tick);
            const int32_t e = (int32_t)(STORE_LAT ? entry_s(v) : entry_e(v));
            rd = strict ? (res > e) : (res >= e);
        }
        const unsigned m = __ballot_sync(0xffffffffu, rd);
        const int run = (m == 0xffffffffu) ? 32 : (__ffs(~m) - 1);
        k += run;
        if (run < 32) break;
    }
    return min(k, lim);
}

// Context of sub-trace b: every instruction still in the simulator, newest
// first: the processor queue, then the memory write queue (whose stores all
// retired from the processor queue, so they are older).
__device__ __forceinline__ int ctx_len(const StepArgs *__restrict__ A, int b) {
    return A->qlen[b] + (A->mlen ? A->mlen[b] : 0);
}
// Entry of context row r (1 <= r <= ctx_len).
__device__ __forceinline__ uint64_t ctx_entry(const StepArgs *__restrict__ A, int b, int r) {
    const int cap = A->cap, ql = A->qlen[b];
    if (r <= ql) {
        int idx = A->qstart[b] + ql - r;
        if (idx >= cap) idx -= cap;
        return A->ring[(size_t)b * cap + idx];
    }
    const int ml = A->mlen[b];
    int idx = A->mstart[b] + ml - (r - ql);
    if (idx >= cap) idx -= cap;
    return A->mring[(size_t)b * cap + idx];
}

// One element of the context gather: thread `gid` of (slot, row, 16-byte chunk).
// Row 0 = current instruction, row j = j-th newest queue entry, rows past the
// queue length are zero, and an inactive slot (sub-trace finished) gets zero rows.
template <typename T>
__device__ __forceinline__ void gather_elem(const StepArgs *__restrict__ A, T *__restrict__ X, int64_t gid) {
    constexpr int V = Vec<T>::N, CH = kNFP / V;
    const int W = A->window;
    const int chunk = (int)(gid % CH);
    const int64_t rowid = gid / CH;
    const int r = (int)(rowid % W);
    const int slot = (int)(rowid / W);
    float v[V];
#pragma unroll
    for (int j = 0; j < V; j++) v[j] = 0.f;
    if (slot < *A->n_active) {
        const int b = A->active[slot];
        const int64_t o = A->offsets[b], n = A->offsets[b + 1] - o;
        const int p = A->pos[b];
        if (p < n) {
            const uint32_t cur = A->records[o + p];
            if (r == 0) {
#pragma unroll
                for (int j = 0; j < V; j++) v[j] = feature(chunk * V + j, cur, cur, false, 0, 0, 0);
            } else if (r <= ctx_len(A, b)) {
                const uint64_t ent = ctx_entry(A, b, r);
                const int32_t res = entry_res(ent, A->tick[b]);
                const uint32_t rec = entry_rec(ent), e = entry_e(ent), sl = entry_s(ent);
#pragma unroll
                for (int j = 0; j < V; j++) v[j] = feature(chunk * V + j, rec, cur, true, res, e, sl);
            }
        }
    }
    store16<T>(X + rowid * kNFP + chunk * V, v);
}

// Bytes of one staged row: a 64-channel row plus 16 bytes of padding, so that
// lanes writing whole rows to shared memory do not collide on banks.
template <typename T> __host__ __device__ constexpr int stage_row_bytes() { return kNFP * (int)sizeof(T) + 16; }

// Copy n (<= 32) staged rows to X rows row0.. with every store instruction
// covering whole contiguous rows (U lanes per row).
template <typename T>
__device__ __forceinline__ void flush_rows(const uint8_t *__restrict__ stg, T *__restrict__ X, int64_t row0, int n,
                                           int lane) {
    constexpr int RB = kNFP * (int)sizeof(T), SR = stage_row_bytes<T>(), U = RB / 16, RPP = 32 / U;
    const int rr = lane / U, u = lane % U;
    uint8_t *g = reinterpret_cast<uint8_t *>(X) + row0 * RB + u * 16;
#pragma unroll 4
    for (int pass = 0; pass < U; pass++) {
        const int r = pass * RPP + rr;
        if (r < n) *reinterpret_cast<uint4 *>(g + (int64_t)r * RB) = *reinterpret_cast<const uint4 *>(stg + r * SR + u * 16);
    }
}

// One row of the context gather, built into `dst` (row 0 = current instruction,
// row j = j-th newest queue entry; rows past the queue length and rows of an
// inactive slot are zero).
template <typename T>
__device__ __forceinline__ void gather_row_into(const StepArgs *__restrict__ A, int64_t rowid, T *dst) {
    const int W = A->window;
    const int r = (int)(rowid % W);
    const int slot = (int)(rowid / W);
    if (slot < *A->n_active) {
        const int b = A->active[slot];
        const int64_t o = A->offsets[b], n = A->offsets[b + 1] - o;
        const int p = A->pos[b];
        if (p < n) {
            const uint32_t cur = A->records[o + p];
            if (r == 0) {
                write_row<T>(dst, cur, cur, false, 0, 0, 0);
                return;
            }
            if (r <= ctx_len(A, b)) {
                const uint64_t ent = ctx_entry(A, b, r);
                write_row<T>(dst, entry_rec(ent), cur, true, entry_res(ent, A->tick[b]), entry_e(ent), entry_s(ent));
                return;
            }
        }
    }
    zero_row_bytes(dst, kNFP * (int)sizeof(T));
}

// A warp gathers rows row0 .. row0+31 (< total) through its staging buffer.
template <typename T>
__device__ __forceinline__ void gather_rows_warp(const StepArgs *__restrict__ A, T *__restrict__ X, int64_t row0,
                                                 int64_t total, uint8_t *__restrict__ stg, int lane) {
    const int n = (int)min((int64_t)32, total - row0);
    if (lane < n) gather_row_into<T>(A, row0 + lane, reinterpret_cast<T *>(stg + lane * stage_row_bytes<T>()));
    __syncwarp();
    flush_rows<T>(stg, X, row0, n, lane);
    __syncwarp();
}

// Pair-major feature tile (the persistent kernel's layout): row r of slot s is
// the half (r & 1) of row ((r >> 1) * Bs + s) of a [W/2 * Bs][2 * 64] array, so
// the two rows a k=2/stride-2 convolution combines are one contiguous K run.
template <typename T>
__device__ __forceinline__ T *pm_row(T *X, int Bs, int slot, int r) {
    return X + ((size_t)(r >> 1) * Bs + slot) * (2 * kNFP) + (size_t)(r & 1) * kNFP;
}

// Store n staged rows (row ids row0.., slot-major over W rows per slot) into
// the pair-major tile, U lanes per row.
template <typename T>
__device__ __forceinline__ void flush_rows_pm(const uint8_t *__restrict__ stg, T *__restrict__ X, int Bs, int W,
                                              int64_t row0, int n, int lane) {
    constexpr int RB = kNFP * (int)sizeof(T), SR = stage_row_bytes<T>(), U = RB / 16, RPP = 32 / U;
    const int rr = lane / U, u = lane % U;
#pragma unroll 4
    for (int pass = 0; pass < U; pass++) {
        const int r = pass * RPP + rr;
        if (r < n) {
            const int64_t id = row0 + r;
            uint8_t *g = reinterpret_cast<uint8_t *>(pm_row<T>(X, Bs, (int)(id / W), (int)(id % W))) + u * 16;
            *reinterpret_cast<uint4 *>(g) = *reinterpret_cast<const uint4 *>(stg + r * SR + u * 16);
        }
    }
}

// Store n staged rows of one slot (its rows r0 ..) into the pair-major tile, U
// lanes per row (the head's path: no division to recover slot and row).
template <typename T>
__device__ __forceinline__ void flush_slot_rows_pm(const uint8_t *__restrict__ stg, T *__restrict__ X, int Bs,
                                                   int slot, int r0, int n, int lane) {
    constexpr int RB = kNFP * (int)sizeof(T), SR = stage_row_bytes<T>(), U = RB / 16, RPP = 32 / U;
    const int rr = lane / U, u = lane % U;
#pragma unroll 4
    for (int pass = 0; pass < U; pass++) {
        const int r = pass * RPP + rr;
        if (r < n) {
            uint8_t *g = reinterpret_cast<uint8_t *>(pm_row<T>(X, Bs, slot, r0 + r)) + u * 16;
            *reinterpret_cast<uint4 *>(g) = *reinterpret_cast<const uint4 *>(stg + r * SR + u * 16);
        }
    }
}

// Dense gather of 32 rows into the pair-major tile; the lane holding row 0 of
// an active sub-trace raises the batch extent to its queue length + 1.
template <typename T>
__device__ __forceinline__ void gather_rows_warp_pm(const StepArgs *__restrict__ A, T *__restrict__ X, int Bs,
                                                    int64_t row0, int64_t total, uint8_t *__restrict__ stg, int lane,
                                                    int *ext) {
    const int W = A->window;
    const int n = (int)min((int64_t)32, total - row0);
    if (lane < n) {
        const int64_t id = row0 + lane;
        gather_row_into<T>(A, id, reinterpret_cast<T *>(stg + lane * stage_row_bytes<T>()));
        const int slot = (int)(id / W);
        if (id % W == 0 && slot < *A->n_active) {
            const int b = A->active[slot];
            if (A->pos[b] < (int)(A->offsets[b + 1] - A->offsets[b])) atomicMax(ext, ctx_len(A, b) + 1);
        }
    }
    __syncwarp();
    flush_rows_pm<T>(stg, X, Bs, W, row0, n, lane);
    __syncwarp();
}

// Move the stores among the k entries at the processor queue's head (ring,
// start qs) to the memory write queue's tail (mring, start ms, length ml), in
// order; non-stores leave.  Whole warp participates; returns the new ml.
__device__ __forceinline__ int stores_to_write_queue(const uint64_t *__restrict__ ring, int qs, int k,
                                                     uint64_t *__restrict__ mring, int ms, int ml, int cap,
                                                     int lane) {
    for (int i0 = 0; i0 < k; i0 += 32) {
        const int i = i0 + lane;
        uint64_t v = 0;
        bool st = false;
        if (i < k) {
            int idx = qs + i;
            if (idx >= cap) idx -= cap;
            v = ring[idx];
            st = rec_is_store(entry_rec(v));
        }
        const unsigned m = __ballot_sync(0xffffffffu, st);
        if (st) {
            int idx = ms + ml + __popc(m & ((1u << lane) - 1u));
            if (idx >= cap) idx -= cap;
            mring[idx] = v;
        }
        ml += __popc(m);
    }
    __syncwarp();
    return ml;
}

// One warp, one active slot.  FC2 arrives as P partial dot products per output
// (one per FC1 column block) which are summed with the bias; the latencies
// follow by head_latency (softplus, clamp, round; or the hybrid class rule);
// then curTick += F, retire (budget RW*F), evict at capacity, append with
// residence 0; after the last instruction, drain one cycle at a time (budget
// RW) and write the sub-trace's cycle count.  With the store latency (NO = 3
// or 33) retired stores move to the memory write queue, which retires in order
// with no bandwidth limit once a residence reaches S; both queues together hold
// at most cap entries and a full simulator evicts its oldest instruction (the
// write queue's head first).  Otherwise the warp writes the slot's feature
// rows for the next step (the gather, fused here); `sq` is this warp's
// shared-memory scratch of 256 queue entries.
// With `pm_slots` > 0 the feature tile is pair-major over that many slots:
// only rows 0 .. max(old, new context length) are written (rows past the
// context are kept zero) and `*ext`, the caller's running maximum of the next
// step's batch extent (a register of the calling warp, which publishes it once),
// is raised to the new context length + 1.
// What the head of one slot reads before any arithmetic of its own: the
// sub-trace, its state and (regression head) this lane's share of the FC2
// partial sums.  Loaded one slot ahead by head phases that walk many slots, so
// that the device-memory round trips overlap the previous slot's work.
struct HeadState {
    int b;
    int64_t o, n;
    int p, tick, qs, ql, ms, ml;
    float zf, ze;   // NO = 2: this lane's sums of the partials i = lane, lane + 32, ...
};
template <int NO>
__device__ __forceinline__ void head_load(const StepArgs *__restrict__ A, int slot, int b, int lane,
                                          const float *__restrict__ part, int P, int part_stride, HeadState &h) {
    h.b = b;
    h.o = A->offsets[b];
    h.n = A->offsets[b + 1] - h.o;
    h.p = A->pos[b];
    h.tick = A->tick[b];
    h.qs = A->qstart[b];
    h.ql = A->qlen[b];
    h.ms = 0;
    h.ml = 0;
    if constexpr (out_lat<NO>() == 3) {
        h.ms = A->mstart[b];
        h.ml = A->mlen[b];
    }
    h.zf = 0.f;
    h.ze = 0.f;
    if constexpr (NO == 2) {
        for (int i = lane; i < P; i += 32) {
            const float2 v = reinterpret_cast<const float2 *>(part)[(size_t)i * part_stride + slot];
            h.zf += v.x;
            h.ze += v.y;
        }
    }
}

template <typename T, int NO = 2>
__device__ __forceinline__ void head_update_state(const StepArgs *__restrict__ A, int slot, int lane, const HeadState &h,
                                                  const float *__restrict__ part, int P, int part_stride,
                                                  const float *__restrict__ b2, T *__restrict__ X,
                                                  uint64_t *__restrict__ sq, uint8_t *__restrict__ stg,
                                                  int pm_slots, int *ext);

template <typename T, int NO = 2>
__device__ __forceinline__ void head_update_warp(const StepArgs *__restrict__ A, int slot, int lane,
                                                 const float *__restrict__ part, int P, int part_stride,
                                                 const float *__restrict__ b2, T *__restrict__ X,
                                                 uint64_t *__restrict__ sq, uint8_t *__restrict__ stg,
                                                 int pm_slots = 0, int *ext = nullptr) {
    HeadState h;
    head_load<NO>(A, slot, A->active[slot], lane, part, P, part_stride, h);
    head_update_state<T, NO>(A, slot, lane, h, part, P, part_stride, b2, X, sq, stg, pm_slots, ext);
}

template <typename T, int NO>
__device__ __forceinline__ void head_update_state(const StepArgs *__restrict__ A, int slot, int lane, const HeadState &h,
                                                  const float *__restrict__ part, int P, int part_stride,
                                                  const float *__restrict__ b2, T *__restrict__ X,
                                                  uint64_t *__restrict__ sq, uint8_t *__restrict__ stg,
                                                  int pm_slots, int *ext) {
    constexpr int NL = out_lat<NO>();
    constexpr bool SQ = NL == 3;
    const int b = h.b;
    const int64_t o = h.o, n = h.n;
    int p = h.p;
    if (p >= n) return;
    // the records of this step's append and of the next step's row 0, and (processor queue
    // of at most 32 entries, no write queue) the whole queue, newest first in the lanes:
    // the retire scan and the next step's rows both come from these registers, so the ring
    // is read once, before the head's arithmetic
    const uint32_t rec_cur = A->records[o + p];
    const uint32_t rec_next = (p + 1 < n) ? A->records[o + p + 1] : 0u;
    const int cap = A->cap, RW = A->retire_width, strict = A->strict;
    uint64_t *ring = A->ring + (size_t)b * cap;
    const bool small = !SQ && h.ql <= 32;
    uint64_t qv = 0;
    if (small && lane < h.ql) {
        int idx = h.qs + h.ql - 1 - lane;
        if (idx >= cap) idx -= cap;
        qv = ring[idx];
    }
    float z[NO];
    if constexpr (NO == 2) {
        z[0] = warp_sum(h.zf) + b2[0];
        z[1] = warp_sum(h.ze) + b2[1];
    } else {
        head_sum_warp<NO>(part, P, part_stride, slot, b2, lane, z);
    }
    float pre[3];
    uint32_t lat[3];
    lat[0] = head_latency<NO, 0>(z, pre[0]);
    lat[1] = head_latency<NO, 1>(z, pre[1]);
    pre[2] = 0.f;
    lat[2] = 0;
    if constexpr (SQ) lat[2] = head_latency<NO, 2>(z, pre[2]);
    const int64_t gi = o + p;
    if (A->replay)
#pragma unroll
        for (int t = 0; t < NL; t++) lat[t] = A->replay[NL * gi + t];
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < NL; t++) {
            if (A->pre_log) A->pre_log[NL * gi + t] = pre[t];
            if (A->lat_log) A->lat_log[NL * gi + t] = (uint8_t)lat[t];
        }
    }
    const uint32_t F = lat[0], E = lat[1], S = lat[2];
    uint64_t *mring = SQ ? A->mring + (size_t)b * cap : nullptr;
    int qs = h.qs, ql = h.ql, ev = 0;
    int ms = h.ms, ml = h.ml;
    const int ctx_old = ql + ml;
    const int ql_old = ql;
    int32_t tick = h.tick + (int32_t)F;
    // processor queue, then (stores) the memory write queue
    auto retire_both = [&](int budget) {
        const int k = retire_run(ring, cap, qs, min(ql, budget), tick, strict, lane);
        if constexpr (SQ) ml = stores_to_write_queue(ring, qs, k, mring, ms, ml, cap, lane);
        qs += k;
        if (qs >= cap) qs -= cap;
        ql -= k;
        if constexpr (SQ) {
            const int km = retire_run<true>(mring, cap, ms, ml, tick, strict, lane);
            ms += km;
            if (ms >= cap) ms -= cap;
            ml -= km;
        }
    };
    if (small) {
        // the oldest-first run of ready entries, from the registers (entry k of the queue
        // is in lane ql - 1 - k)
        const int lim = min(ql, RW * (int)F);
        const uint64_t v = __shfl_sync(0xffffffffu, qv, max(ql - 1 - lane, 0));
        bool rd = false;
        if (lane < lim) {
            const int32_t res = entry_res(v, tick), e = (int32_t)entry_e(v);
            rd = strict ? (res > e) : (res >= e);
        }
        const unsigned m = __ballot_sync(0xffffffffu, rd);
        const int k = min((m == 0xffffffffu) ? 32 : (__ffs(~m) - 1), lim);
        qs += k;
        if (qs >= cap) qs -= cap;
        ql -= k;
    } else {
        retire_both(RW * (int)F);
    }
    if (ql + ml == cap) {  // full: drop the oldest instruction
        if (ml > 0) {
            ms = (ms + 1 == cap) ? 0 : ms + 1;
            ml--;
        } else {
            qs = (qs + 1 == cap) ? 0 : qs + 1;
            ql--;
        }
        ev = 1;
    }
    const uint64_t appended = pack_entry(rec_cur, E, S, (uint32_t)tick);
    if (lane == 0) {
        int idx = qs + ql;
        if (idx >= cap) idx -= cap;
        ring[idx] = appended;
    }
    ql++;
    p++;
    __syncwarp();
    if (p == n) {  // drain: Delta of Eq. 1
        while (ql + ml > 0) {
            tick += 1;
            retire_both(RW);
        }
        if (lane == 0) A->cycles_out[b] = tick;
    } else if (X) {
        // next step's input rows of this slot: row 0 = instruction p, row r = r-th newest
        // context entry.  The context is copied newest-first into shared memory with
        // independent loads first (or, for a small queue, from the registers read at the
        // start: row 1 is the entry just appended, row r >= 2 the old (r - 2)-th newest).
        if (small) {
            if (lane == 0) sq[1] = appended;
            if (lane + 2 <= ql && lane < ql_old) sq[lane + 2] = qv;
        } else {
            for (int r = lane + 1; r <= ql + ml; r += 32) {
                int idx;
                if (r <= ql) {
                    idx = qs + ql - r;
                    if (idx >= cap) idx -= cap;
                    sq[r] = ring[idx];
                } else {
                    idx = ms + ml - (r - ql);
                    if (idx >= cap) idx -= cap;
                    sq[r] = mring[idx];
                }
            }
        }
        __syncwarp();
        const int W = A->window;
        const uint32_t cur = rec_next;
        constexpr int SR = stage_row_bytes<T>();
        const int ctx_new = ql + ml;
        const int rows = pm_slots > 0 ? min(W, max(ctx_old, ctx_new) + 1) : W;
        if (pm_slots > 0) *ext = max(*ext, ctx_new + 1);   // the caller's running maximum
        for (int r0 = 0; r0 < rows; r0 += 32) {   // a lane builds a row, the warp stores rows whole
            const int r = r0 + lane;
            T *row = reinterpret_cast<T *>(stg + lane * SR);
            if (r < rows) {
                if (r == 0) {
                    write_row<T>(row, cur, cur, false, 0, 0, 0);
                } else if (r <= ctx_new) {
                    const uint64_t ent = sq[r];
                    write_row<T>(row, entry_rec(ent), cur, true, entry_res(ent, tick), entry_e(ent), entry_s(ent));
                } else {
                    zero_row_bytes(row, kNFP * (int)sizeof(T));
                }
            }
            __syncwarp();
            if (pm_slots > 0)
                flush_slot_rows_pm<T>(stg, X, pm_slots, slot, r0, min(32, rows - r0), lane);
            else
                flush_rows<T>(stg, X, (int64_t)slot * W + r0, min(32, rows - r0), lane);
            __syncwarp();
        }
    }
    if (lane == 0) {
        A->tick[b] = tick;
        A->pos[b] = p;
        A->qstart[b] = qs;
        A->qlen[b] = ql;
        if (ev) A->evict[b] += ev;   // rare: a read-modify-write only when it changes
        if constexpr (SQ) {
            A->mstart[b] = ms;
            A->mlen[b] = ml;
        }
    }
}

// Stable in-place compaction of the active list, one block (any size that is a
// multiple of 32, at most 1024): drop finished sub-traces so the batch stays dense.
__device__ __forceinline__ void compact_block(const StepArgs *__restrict__ A) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int n = *A->n_active;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        int b = -1;
        bool keep = false;
        if (i < n) {
            b = A->active[i];
            keep = A->pos[b] < (int)(A->offsets[b + 1] - A->offsets[b]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        const int pre = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        if (w == 0) {
            int v = lane < nw ? wsum[lane] : 0, x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < nw) wsum[lane] = x - v;  // exclusive prefix over warps
        }
        __syncthreads();
        const int dst = base + wsum[w] + pre;
        if (keep) A->active[dst] = b;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base = dst + (keep ? 1 : 0);
        __syncthreads();
    }
    if (threadIdx.x == 0) *A->n_active = base;
}

}  // namespace simnet
