// common.cuh -- types shared by libsimnet's translation units (device side and host side).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "simnet.h"

namespace simnet {

constexpr int kNF = SIMNET_N_FEATURES;  // real features per row (Sec. 2.2)
constexpr int kNFP = 64;                // features per row in device layout (zero padded)
constexpr int kMaxConv = 8;
constexpr int kMaxGemm = 3 * kMaxConv + 1;  // GEMMs of the deepest CNN: 3 per residual block + FC1
constexpr int kOutHybrid = 22;          // FC2 outputs of the hybrid head: per latency 10 class logits + 1 value

// Device status word values (written by kernels, read by the host after a call).
enum : int32_t { kStatusOk = 0, kStatusTimeout = 1, kStatusBadTrace = 2 };

// Ring entry of the processor queue and the memory write queue: record (26 bits)
// | E (8 bits) << 26 | S (8 bits) << 34 | fetch tick mod 2^22 << 42.  A
// residence never comes near 2^22 cycles (an entry is at most 255 cycles from
// its fetch to its latency, and then leaves within cap / retire_width further
// cycles of retire bandwidth and one more jump of at most 255), so
// (curTick - stored tick) mod 2^22 is the residence exactly.
constexpr uint32_t kTickMask = (1u << 22) - 1u;
__host__ __device__ __forceinline__ uint64_t pack_entry(uint32_t rec, uint32_t e, uint32_t s, uint32_t tick) {
    return (uint64_t)(rec & 0x3ffffffu) | ((uint64_t)(e & 0xffu) << 26) | ((uint64_t)(s & 0xffu) << 34) |
           ((uint64_t)(tick & kTickMask) << 42);
}
__host__ __device__ __forceinline__ uint32_t entry_rec(uint64_t v) { return (uint32_t)(v & 0x3ffffffu); }
__host__ __device__ __forceinline__ uint32_t entry_e(uint64_t v) { return (uint32_t)((v >> 26) & 0xffu); }
__host__ __device__ __forceinline__ uint32_t entry_s(uint64_t v) { return (uint32_t)((v >> 34) & 0xffu); }
// residence of an entry at curTick `tick`
__host__ __device__ __forceinline__ int32_t entry_res(uint64_t v, int32_t tick) {
    return (int32_t)(((uint32_t)tick - (uint32_t)(v >> 42)) & kTickMask);
}
__host__ __device__ __forceinline__ bool rec_is_store(uint32_t rec) { return (rec >> 21) & 1u; }

// Everything a step's simulation kernels need; lives in device memory so that a
// captured CUDA graph stays valid when the caller passes new trace buffers.
struct StepArgs {
    // the call
    const uint32_t *records;
    const int64_t *offsets;
    int64_t *cycles_out;
    uint8_t *lat_log;
    float *pre_log;
    const uint8_t *replay;
    // per-sub-trace state [B]
    int32_t *tick;
    int32_t *pos;
    int32_t *qstart;
    int32_t *qlen;
    int32_t *evict;
    uint64_t *ring;  // [B][cap]
    // batch slots
    int32_t *active;    // [B] slot -> sub-trace
    int32_t *n_active;  // [1]
    int32_t *status;    // [1]
    // shapes
    int32_t n_sub;
    int32_t window;
    int32_t cap;
    int32_t retire_width;
    int32_t strict;
    int32_t hidden;
    // memory write queue (Sec. 3.2), with the store latency as a third latency;
    // null when it is not modelled
    int32_t *mstart;  // [B]
    int32_t *mlen;    // [B]
    uint64_t *mring;  // [B][cap]
    int32_t n_lat;    // latencies per instruction: 2 (F, E) or 3 (F, E, S)
};

// Workspace buffers a GEMM of the CNN reads or writes (see GemmLayer).
enum GemmBuf : int { kBufNone = -1, kBufX = 0, kBufAct0 = 1, kBufAct1 = 2, kBufTmpA = 3, kBufTmpS = 4, kBufH1 = 5 };

// A GEMM layer C[M, N] = act(A[M, K] * B[N, K]^T * scale + bias [+ R]), M = n_active * m_mult.
struct GemmLayer {
    int m_mult;    // output rows per sub-trace
    int K;         // reduction length (padded)
    int N;         // output columns
    int relu;
    int in_buf = kBufX, out_buf = kBufH1;  // A and C
    int res_buf = kBufNone;  // R [M][N] in the layer precision, added before the activation
    int kind = 0;            // timing kind offset (conv layer / residual block index; FC1 last)
    const void *B; // weights [N][K] in the layer's precision
    const float *bias;   // [N]
    const float *scale;  // [N] per-output-channel dequant scale (FP8) or nullptr
    const float *oscale; // [N] multiplier applied before storing (FP8 requant) or nullptr
};

// ------------------------------------------------------------------ feature encoding (Sec. 2.2)
// Channel c of a row.  `rec` is the row's instruction; for a context row (ctx)
// `cur` is the instruction being predicted, `res` its residence, `e` its
// execution and `s` its store latency.  Layout: 0-31 opcode one-hot; 32-34
// src0/src1/dst / 32; 35-37 load/store/branch; 38-40 cache-level one-hot;
// 41 mispredict; 42 min(res,4095)/64; 43 E/64; 44 S/64 for a store (0 without
// the memory write queue, whose entries carry S = 0); 45-47 rec.dst equals
// cur.src0/src1/dst; 48 both memory ops at one cache level; 49-63 zero.
__device__ __forceinline__ float feature(int c, uint32_t rec, uint32_t cur, bool ctx, int32_t res,
                                         uint32_t e, uint32_t s) {
    if (c < 32) return (rec & 31u) == (uint32_t)c ? 1.f : 0.f;
    const uint32_t dst = (rec >> 15) & 31u;
    switch (c) {
        case 32: return (float)((rec >> 5) & 31u) * 0.03125f;
        case 33: return (float)((rec >> 10) & 31u) * 0.03125f;
        case 34: return (float)dst * 0.03125f;
        case 35: return (float)((rec >> 20) & 1u);
        case 36: return (float)((rec >> 21) & 1u);
        case 37: return (float)((rec >> 22) & 1u);
        case 38: case 39: case 40: return ((rec >> 23) & 3u) == (uint32_t)(c - 38) ? 1.f : 0.f;
        case 41: return (float)((rec >> 25) & 1u);
        case 42: return ctx ? (float)min(res, 4095) * 0.015625f : 0.f;
        case 43: return ctx ? (float)e * 0.015625f : 0.f;
        case 44: return (ctx && rec_is_store(rec)) ? (float)s * 0.015625f : 0.f;
        case 45: return (ctx && dst == ((cur >> 5) & 31u)) ? 1.f : 0.f;
        case 46: return (ctx && dst == ((cur >> 10) & 31u)) ? 1.f : 0.f;
        case 47: return (ctx && dst == ((cur >> 15) & 31u)) ? 1.f : 0.f;
        case 48: {
            const bool m0 = (rec >> 20) & 3u, m1 = (cur >> 20) & 3u;  // load or store
            return (ctx && m0 && m1 && ((rec >> 23) & 3u) == ((cur >> 23) & 3u)) ? 1.f : 0.f;
        }
        default: return 0.f;
    }
}


// Launch a kernel, optionally as a programmatic dependent launch: it may start
// while the previous kernel in the stream finishes; every kernel of this
// library executes griddepcontrol.wait before touching data other kernels write.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

}  // namespace simnet
