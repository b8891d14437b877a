// persist.cu -- the whole lock-step simulation of one simnet_simulate call in a
// single persistent, cooperative kernel (one CTA per SM).
//
// Every step runs as phases separated by grid-wide barriers:
//   GEMM phase per CNN layer (Sec. 2.3): the layer's 128-row tiles are spread
//     over the CTAs; inside a CTA the roles of the tensor-core GEMM kernel work
//     as usual (warp 0 TMA producer, warp 1 tcgen05.mma issuer, warps 2-9
//     TMEM epilogue) and their pipeline counters carry over from phase to
//     phase, so the shared-memory ring, mbarriers and TMEM (allocated once)
//     stay in use for the whole call;
//   head phase: every warp of the grid takes active sub-traces: FC2 from the
//     FC1 epilogue's partial sums, softplus/round, clock and queue update,
//     drain, and the feature rows of the next step (Sec. 3.2, Eq. 1);
//   every `compact_every` steps (uneven lengths): CTA 0 compacts the active
//     list, then all threads re-gather the feature tile.
// Padding extent: rows past every queue are zero features, so each conv layer
// maps them to one constant row (per layer) and FC1 sees that constant at every
// padded position.  The kernel therefore computes, each step, only the row
// positions below the batch extent e (the longest queue + 1, rounded up to a
// whole conv-output row), and FC1's epilogue adds S[e], the precomputed FC1
// contribution of the constant rows at positions >= e.  Activations are stored
// pair-major ([row pair][slot][2C]) so that the two rows a k=2/stride-2
// convolution combines are one contiguous K run of a 2D TMA box.
// The barrier is a monotone counter with release/acquire at GPU scope and a
// bounded spin; on expiry the kernel records a timeout, every CTA leaves the
// step loop, frees TMEM and returns.  Stores that a later TMA load reads are
// followed by a generic-to-async proxy fence.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>

#include "ctx.cuh"
#include "sim_device.cuh"
#include "tc_ptx.cuh"

namespace simnet {

struct PLayer {
    CUtensorMap tA, tB;  // A: pair-major input [pairs * B][2 * C_in]; B: weights [N][K]
    const float *bias, *scale, *oscale;
    void *out;           // pair-major activations [pairs * B][2N], or FC2 partials [2*N/BN][B][n_out] float
    int K, N, BN, out_part, n_tiles_n;
    int cin;             // input row width in elements (FC1: channels of one input row)
    int pos_shift;       // conv: output positions computed = e << pos_shift
    int relu;            // activation after bias (and shortcut)
    // Pointwise GEMM of a residual block: its rows are output positions.  The
    // pair-major [pairs * B][2N] tile is read and written as [2 * pairs * B][N]
    // (row 2 * (pair * B + slot) + half), which is the pair-major layout of the
    // block output again; `resid` (the block's shortcut, same view) is added
    // before the activation.  Tiles take one pair of 64 slots (128 rows).
    int rows_plain;
    const void *resid;
    int kind;            // timing kind offset: conv layer or residual block index, FC1 last
    // per-layer extent: output position p covers input rows [p << pos_log, (p + 1) << pos_log)
    // of the window; positions at or past ceil(extent / 2^pos_log) see only padding rows and
    // hold the constant row `cst` (storage units [N]); rows_out = the layer's positions
    int pos_log, rows_out;
    const float *cst;
    int pair_next;       // layer l + 1 (same input, K and N) runs in this layer's phase
    int prm_off;         // this layer's parameters in shared memory (staged once per call):
                         // bias [N], FP8 scale [N] and requant [N], FC1 with 2 outputs: FC2 rows [2N]
};

struct PArgs {
    PLayer layer[kMaxGemm];
    const StepArgs *A;
    void *X;
    const float *part;
    const float *w2, *b2;
    const float *fc1_const;       // [rows_n + 1][H]
    int *ext;                     // [2] batch extent per step parity
    unsigned *bar_counter;        // zero at launch
    int *abort_g;                 // zero at launch
    int32_t *status;
    unsigned long long *phase_ns; // [SIMNET_KERNEL_KINDS] summed phase times (CTA 0), or null
    unsigned long long *phase_n;  // [SIMNET_KERNEL_KINDS] phase counts
    unsigned long long *exec;     // [layer] GEMM rows computed over the steps, on request: output
                                  // positions x active slots (FC1: last-layer positions x slots)
    unsigned long long *detail;   // [kMaxConv+1][4] CTA 0, ns after each GEMM phase starts: first data,
                                  // last MMA commit, epilogue done, barrier passed (or null)
    int64_t n_steps;
    int64_t spin_ns;
    int64_t bar_spin_ns;          // grid-barrier wait bound
    int n_layers, B, P, compact_every, stages, stage_bytes, prm_floats;
    int n_conv;                   // conv layers or residual blocks (the pair-major extent's halvings)
    int w2h_off;                  // hybrid / store heads: per-epilogue-warp FC2 row slices at prm + w2h_off
    int cst_off;                  // FC1's padding row S[e] of the current step at prm + cst_off
    int rows_n, e_round;          // last conv rows; FC1 k-block rows (extent granularity)
    // Fused first two conv layers (plain CNN, 256 channels): one phase computes each tile
    // of 128 slots at one output position of conv2 from conv1's two positions under it;
    // conv1's output goes from its accumulator into tensor memory as conv2's A operand
    // and never reaches device memory.
    int fuse, fu;                 // fused phase on; its operand units (16 KB each) in the stage ring
    int ring_bytes;               // shared memory before the barrier area: the stage ring, or the
                                  // fused phase's units and resident weights where they need more
    CUtensorMap tW1, tW2h;        // conv1's and conv2's weights in 128-row boxes
};

namespace {
using namespace tcx;

constexpr int kThreads = 320, kWarps = 10, kEpiWarps = 8;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier; false when the kernel is aborting (timeout here or elsewhere).
__device__ bool grid_sync(const PArgs &a, unsigned &target, volatile int *cta_abort) {
    asm volatile("fence.proxy.async;" ::: "memory");   // generic writes (global and shared) before async-proxy use
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*cta_abort) atomicExch(a.abort_g, 1);   // a bounded wait in this CTA gave up: stop everyone
        target += gridDim.x;
        __threadfence();
        atomicAdd(a.bar_counter, 1u);
        const uint64_t t0 = gtimer();
        while (ld_acquire(a.bar_counter) < target) {
            if (*(volatile int *)a.abort_g) { *cta_abort = 1; break; }
            if ((int64_t)(gtimer() - t0) > a.bar_spin_ns) {
                atomicExch(a.abort_g, 1);
                atomicExch(a.status, kStatusTimeout);
                *cta_abort = 1;
                break;
            }
        }
        if (*(volatile int *)a.abort_g) *cta_abort = 1;
    }
    __syncthreads();
    return *cta_abort == 0;
}

// All warps of the grid gather 32-row groups (every row of every slot) into
// the pair-major tile through their staging buffers (the stage ring is free
// between GEMM phases), raising the extent `ext`.
template <typename T>
__device__ void gather_phase(const PArgs &a, uint8_t *ring, int *ext) {
    const int64_t total = (int64_t)a.B * a.A->window;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *stg = ring + warp * (32 * stage_row_bytes<T>());
    for (int64_t row0 = ((int64_t)blockIdx.x * kWarps + warp) * 32; row0 < total;
         row0 += (int64_t)gridDim.x * kWarps * 32)
        gather_rows_warp_pm<T>(a.A, reinterpret_cast<T *>(a.X), a.B, row0, total, stg, lane, ext);
}

// kernel parameters (__grid_constant__) stay under the 32 KB parameter limit
static_assert(sizeof(PArgs) <= 32000, "persistent kernel arguments too large");

struct Pipe {  // pipeline counters that carry over between GEMM phases
    int prod_it = 0, mma_it = 0, mma_tc = 0, epi_tc = 0;
    int res = 0;   // phases that loaded their weights once (resident), for that barrier's parity
    int fprod = 0, fmma = 0, fz = 0, fw1 = 0;   // fused phase: operand units, tiles, weight loads,
    int fpc = 0, fe = 0;                        // pieces issued, pieces drained by this warpgroup
};

// Shared-memory barrier area: S full and S empty stage barriers, two accumulator
// full and two empty barriers, the TMEM address and abort flag, the resident-weight
// barrier; from kFuBar(S): the fused phase's unit full / empty barriers, its four
// A-operand quarters and its resident-weight barrier.
constexpr int kBarBytes = 512;
__host__ __device__ constexpr int kFuBar(int S) { return 2 * S + 6; }

// Positions [lo, hi) of every slot below M in a layer's pair-major output tile
// get the layer's constant row; the epilogue warps of the grid share the work.
template <typename T>
__device__ void fill_const(const PArgs &a, const PLayer &L, int lo, int hi, int M) {
    if (lo >= hi) return;
    constexpr int V = Vec<T>::N;
    const int N = L.N, chunks = N / V;
    const int64_t total = (int64_t)(hi - lo) * M * chunks;
    const int64_t nth = (int64_t)gridDim.x * 32 * kEpiWarps;
    for (int64_t i = (int64_t)blockIdx.x * 32 * kEpiWarps + (threadIdx.x - 64); i < total; i += nth) {
        const int ch = (int)(i % chunks);
        const int64_t r = i / chunks;
        const int slot = (int)(r % M), pos = lo + (int)(r / M);
        float v[V];
#pragma unroll
        for (int j = 0; j < V; j++) v[j] = L.cst[ch * V + j];
        T *dst = reinterpret_cast<T *>(L.out) + ((size_t)(pos >> 1) * a.B + slot) * 2 * N + (size_t)(pos & 1) * N +
                 ch * V;
        store16<T>(dst, v);
    }
}

// One GEMM phase: the tiles of layer l, or of layers l and l2 together (a residual
// block's conv and projection: same input and shape, independent outputs, so one
// phase and one grid barrier serve both; tiles [0, T0) are layer l's).
template <bool FP8, int NO>
__device__ uint64_t gemm_phase(const PArgs &a, int l, int l2, int e, int n_now, int n_prev, uint8_t *smem,
                               uint64_t *bars, float *prm, uint8_t *staging, uint32_t tmem_base,
                               volatile int *cta_abort, Pipe &pp, bool rev) {
    const PLayer &L = a.layer[l];
    constexpr int BK = FP8 ? 128 : 64;
    const int S = a.stages, N = L.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // parameters were staged at the start of the call; only FC1's padding row changes per step
    float *s_bias = prm + L.prm_off;
    float *s_w2 = s_bias + (FP8 ? 3 * N : N), *s_cst = prm + a.cst_off;
    if (L.out_part) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) s_cst[i] = a.fc1_const[(size_t)e * N + i];
        __syncthreads();
    }
    const uint32_t smem_base = smem_u32(smem);
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[S + s]); };
    auto tfull = [&](int x) { return smem_u32(&bars[2 * S + x]); };
    auto tempty = [&](int x) { return smem_u32(&bars[2 * S + 2 + x]); };
    const int M = min(*a.A->n_active, a.B);                 // slots
    const int n_sb = L.rows_plain ? (M + BM / 2 - 1) / (BM / 2) : (M + BM - 1) / BM;   // slot blocks per tile
    int n_pos = L.out_part ? 1 : n_now;                     // output row positions computed
    if (L.rows_plain) n_pos = (n_pos + 1) >> 1;             // ... as pairs of positions
    const int T0 = n_pos * n_sb * L.n_tiles_n;
    const int n_tiles = T0 + (l2 >= 0 ? n_pos * n_sb * a.layer[l2].n_tiles_n : 0);
    const int KB = L.out_part ? e * L.cin / BK : L.K / BK;   // the paired layer has the same K
    // Consecutive phases walk their tiles in opposite orders, so a phase starts on the
    // input the previous one wrote last, which is likeliest still in L2.
    auto vt = [&](int t) { return rev ? n_tiles - 1 - t : t; };
    if (a.exec && blockIdx.x == 0 && threadIdx.x == 0) {   // the padding extent's saving, counted
        const unsigned long long rows = (unsigned long long)(L.out_part ? e : n_now) * (unsigned long long)M;
        atomicAdd(&a.exec[l], rows);
        if (l2 >= 0) atomicAdd(&a.exec[l2], rows);
    }
    // tile t -> its layer (0: l, 1: l2), input position (pair), slot block, column block
    auto tile_of = [&](int t, int &which, int &pos, int &sb, int &nt) {
        which = (!FP8 && t >= T0) ? 1 : 0;   // residual blocks (the only pairs) are BF16
        if (which) t -= T0;
        const int ntn = which ? a.layer[l2].n_tiles_n : L.n_tiles_n;
        nt = t % ntn;
        const int r = t / ntn;
        sb = r % n_sb;
        pos = r / n_sb;
    };
    const int64_t lim = a.spin_ns;
    const bool det = a.detail && blockIdx.x == 0;
    const uint64_t t_phase = det ? gtimer() : 0;
    // A layer whose whole weight matrix (one column block of KB panels) fits beside S
    // operand-only stages keeps it in shared memory for the phase, loaded once: the first
    // conv layer (K = 128, two panels) would else reload its 64 KB for every 128-row tile.
    const bool resident = !L.out_part && l2 < 0 && L.n_tiles_n == 1 && blockIdx.x < n_tiles &&
                          (uint32_t)S * A_BYTES + (uint32_t)KB * L.BN * ROW_BYTES <= (uint32_t)S * a.stage_bytes;
    const uint32_t res_base = smem_base + (uint32_t)S * A_BYTES, res_panel = (uint32_t)L.BN * ROW_BYTES;
    const uint32_t bres = smem_u32(&bars[2 * S + 5]);
    auto a_stage = [&](int s) {
        return resident ? smem_base + (uint32_t)s * A_BYTES : smem_base + (uint32_t)s * a.stage_bytes;
    };
    if (warp == 0) {
        if (lane == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            bool ok = true;
            if (resident) {   // the stages of the previous phase are all consumed (grid barrier)
                mbar_expect_tx(bres, (uint32_t)KB * res_panel);
                for (int kb = 0; kb < KB; kb++) tma_load_2d(res_base + (uint32_t)kb * res_panel, &L.tB, bres, kb * BK, 0);
            }
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                int which, pos, sb, nt;
                tile_of(vt(t), which, pos, sb, nt);
                const PLayer &Lt = which ? a.layer[l2] : L;
                const int n0 = nt * Lt.BN;
                const uint32_t stage_tx = (uint32_t)(A_BYTES + (resident ? 0 : Lt.BN * ROW_BYTES));
                for (int kb = 0; kb < KB; kb++, pp.prod_it++) {
                    const int s = pp.prod_it % S;
                    const uint32_t ph = (uint32_t)(pp.prod_it / S) & 1u;
                    if (!mbar_wait(empty(s), ph ^ 1u, lim, cta_abort, a.status)) { ok = false; break; }
                    const uint32_t sa = a_stage(s);
                    // A: conv -> input pair `pos`; FC1 -> the input row holding this K slice
                    int ax, ay;
                    if (L.out_part) {
                        const int kk = kb * BK, row = kk / L.cin;
                        ax = (row & 1) * L.cin + kk % L.cin;
                        ay = (row >> 1) * a.B + sb * BM;
                    } else if (L.rows_plain) {   // pair `pos`, slots sb * 64 ..: 128 consecutive view rows
                        ax = kb * BK;
                        ay = 2 * (pos * a.B + sb * (BM / 2));
                    } else {
                        ax = kb * BK;
                        ay = pos * a.B + sb * BM;
                    }
                    mbar_expect_tx(full(s), stage_tx);
                    tma_load_2d(sa, &L.tA, full(s), ax, ay);
                    if (!resident) tma_load_2d(sa + A_BYTES, &Lt.tB, full(s), kb * BK, n0);
                }
            }
        }
    } else if (warp == 1) {
        {   // the whole warp runs the issue loop, one elected lane issues (umma_warp)
            bool ok = true;
            if (resident) {
                ok = __all_sync(0xffffffffu, mbar_wait(bres, (uint32_t)pp.res & 1u, lim, cta_abort, a.status));
                pp.res++;
                tc_fence_after();
            }
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, pp.mma_tc++) {
                const uint32_t ID = idesc_rt((!FP8 && vt(t) >= T0) ? a.layer[l2].BN : L.BN, FP8);
                const int acc = pp.mma_tc & 1;
                const uint32_t aph = (uint32_t)(pp.mma_tc >> 1) & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait(tempty(acc), aph ^ 1u, lim, cta_abort, a.status))) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * 256);
                for (int kb = 0; kb < KB; kb++, pp.mma_it++) {
                    const int s = pp.mma_it % S;
                    const uint32_t ph = (uint32_t)(pp.mma_it / S) & 1u;
                    if (!__all_sync(0xffffffffu, mbar_wait(full(s), ph, lim, cta_abort, a.status))) { ok = false; break; }
                    tc_fence_after();
                    if (det && lane == 0 && t == (int)blockIdx.x && kb == 0)
                        atomicAdd(&a.detail[4 * l + 0], gtimer() - t_phase);
                    const uint32_t sa = a_stage(s);
                    const uint64_t ad = sdesc(sa), bd = sdesc(resident ? res_base + (uint32_t)kb * res_panel : sa + A_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        umma_warp<FP8>(d, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), ID, (kb | k) != 0 ? 1u : 0u);
                    umma_commit_warp(empty(s));
                }
                if (ok) umma_commit_warp(tfull(acc));
            }
            if (det && lane == 0) atomicAdd(&a.detail[4 * l + 1], gtimer() - t_phase);
        }
        __syncwarp();
    } else {
        // positions this step no longer computes get the constant row first (the
        // pointwise phase computes whole pairs)
        if (!L.out_part) {
            using T = typename std::conditional<FP8, __nv_fp8_e4m3, __nv_bfloat16>::type;
            fill_const<T>(a, L, L.rows_plain ? (n_now + 1) & ~1 : n_now, n_prev, M);
            if (l2 >= 0) fill_const<T>(a, a.layer[l2], n_now, n_prev, M);
        }
        const int q = warp & 3, half = (warp - 2) >> 2;
        constexpr int OES = FP8 ? 1 : 2;
        constexpr int CB = 32 * OES, SROW = CB + 16;
        uint8_t *stg = staging + (warp - 2) * 32 * SROW;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, pp.epi_tc++) {
            int which, pos, sb, nt;
            tile_of(vt(t), which, pos, sb, nt);
            const PLayer &Lt = which ? a.layer[l2] : L;
            const int BN = Lt.BN, CPW = BN / 64;
            // this tile's layer parameters
            const float *t_bias = prm + Lt.prm_off, *t_scale = t_bias + N, *t_oscale = t_bias + 2 * N;
            const int m0 = L.rows_plain ? 2 * (pos * a.B + sb * (BM / 2)) : sb * BM, n0 = nt * BN;
            const int acc = pp.epi_tc & 1;
            const uint32_t aph = (uint32_t)(pp.epi_tc >> 1) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait(tfull(acc), aph, lim, cta_abort, a.status))) break;
            tc_fence_after();
            const int row = m0 + q * 32 + lane;
            const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 256 + half * (BN / 2));
            float pf = 0.f, pe = 0.f;
            constexpr int NH = NO == 2 ? 1 : NO;
            float ph[NH];
#pragma unroll
            for (int o = 0; o < NH; o++) ph[o] = 0.f;
            for (int c = 0; c < CPW; c++) {
                uint32_t r[32];
                tmem_ld32(tbase + (uint32_t)(c * 32), r);
                const int col0 = n0 + half * (BN / 2) + c * 32;
                float v[32];
                uint32_t rs[16];   // residual block: the shortcut of this row (BF16 pairs, same view)
#pragma unroll
                for (int j = 0; j < 16; j++) rs[j] = 0u;
                if constexpr (!FP8) {
                    if (L.resid && (sb * (BM / 2) + ((q * 32 + lane) >> 1)) < M) {
                        const uint4 *rp = reinterpret_cast<const uint4 *>(
                            reinterpret_cast<const __nv_bfloat16 *>(L.resid) + (size_t)row * N + col0);
#pragma unroll
                        for (int q4 = 0; q4 < 4; q4++) {
                            const uint4 u = rp[q4];
                            rs[4 * q4] = u.x;
                            rs[4 * q4 + 1] = u.y;
                            rs[4 * q4 + 2] = u.z;
                            rs[4 * q4 + 3] = u.w;
                        }
                    }
                }
                if (!L.out_part && !L.resid && Lt.relu) {
                    // a plain conv layer: bias (FP8: and the scales) four columns to a load, no
                    // shortcut (this loop bounded the first layer's phase at c5)
                    const float4 *b4 = reinterpret_cast<const float4 *>(t_bias + col0);
                    const float4 *s4 = reinterpret_cast<const float4 *>(t_scale + col0);
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 bb = b4[j4];
                        float x0 = __uint_as_float(r[4 * j4]), x1 = __uint_as_float(r[4 * j4 + 1]);
                        float x2 = __uint_as_float(r[4 * j4 + 2]), x3 = __uint_as_float(r[4 * j4 + 3]);
                        if constexpr (FP8) {   // scale and bias carry the requant multiplier
                            const float4 sc = s4[j4];
                            v[4 * j4] = fmaxf(x0 * sc.x + bb.x, 0.f);
                            v[4 * j4 + 1] = fmaxf(x1 * sc.y + bb.y, 0.f);
                            v[4 * j4 + 2] = fmaxf(x2 * sc.z + bb.z, 0.f);
                            v[4 * j4 + 3] = fmaxf(x3 * sc.w + bb.w, 0.f);
                        } else {
                            v[4 * j4] = fmaxf(x0 + bb.x, 0.f);
                            v[4 * j4 + 1] = fmaxf(x1 + bb.y, 0.f);
                            v[4 * j4 + 2] = fmaxf(x2 + bb.z, 0.f);
                            v[4 * j4 + 3] = fmaxf(x3 + bb.w, 0.f);
                        }
                    }
                } else if (L.out_part) {
                    // FC1: dequant scale (FP8), the constant rows past the extent, bias, ReLU,
                    // four columns to a load (the general path's order of operations)
                    const float4 *c4 = reinterpret_cast<const float4 *>(s_cst + col0);
                    const float4 *b4 = reinterpret_cast<const float4 *>(t_bias + col0);
                    const float4 *s4 = reinterpret_cast<const float4 *>(t_scale + col0);
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 cc = c4[j4], bb = b4[j4];
                        float x0 = __uint_as_float(r[4 * j4]), x1 = __uint_as_float(r[4 * j4 + 1]);
                        float x2 = __uint_as_float(r[4 * j4 + 2]), x3 = __uint_as_float(r[4 * j4 + 3]);
                        if constexpr (FP8) {
                            const float4 sc = s4[j4];
                            x0 *= sc.x;
                            x1 *= sc.y;
                            x2 *= sc.z;
                            x3 *= sc.w;
                        }
                        x0 = (x0 + cc.x) + bb.x;
                        x1 = (x1 + cc.y) + bb.y;
                        x2 = (x2 + cc.z) + bb.z;
                        x3 = (x3 + cc.w) + bb.w;
                        if (Lt.relu) {
                            x0 = fmaxf(x0, 0.f);
                            x1 = fmaxf(x1, 0.f);
                            x2 = fmaxf(x2, 0.f);
                            x3 = fmaxf(x3, 0.f);
                        }
                        v[4 * j4] = x0;
                        v[4 * j4 + 1] = x1;
                        v[4 * j4 + 2] = x2;
                        v[4 * j4 + 3] = x3;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        float x = __uint_as_float(r[j]);
                        if (FP8) x *= t_scale[col0 + j];
                        if (L.out_part) x += s_cst[col0 + j];   // FC1: the constant rows past the extent
                        // BF16 bits to FP32: the value's 16 bits as the high half of an FP32 word
                        const float rv = __uint_as_float((j & 1) ? (rs[j >> 1] & 0xffff0000u) : (rs[j >> 1] << 16));
                        x += t_bias[col0 + j] + rv;
                        if (Lt.relu) x = fmaxf(x, 0.f);
                        if (FP8 && !L.out_part) x *= t_oscale[col0 + j];
                        v[j] = x;
                    }
                }
                if (L.out_part) {
                    if constexpr (NO == 2) {   // the two FC2 rows four columns to a load
                        const float4 *wa = reinterpret_cast<const float4 *>(s_w2 + col0);
                        const float4 *wb = reinterpret_cast<const float4 *>(s_w2 + N + col0);
#pragma unroll
                        for (int j4 = 0; j4 < 8; j4++) {
                            const float4 fa = wa[j4], fb = wb[j4];
                            pf = fmaf(v[4 * j4], fa.x, pf);
                            pe = fmaf(v[4 * j4], fb.x, pe);
                            pf = fmaf(v[4 * j4 + 1], fa.y, pf);
                            pe = fmaf(v[4 * j4 + 1], fb.y, pe);
                            pf = fmaf(v[4 * j4 + 2], fa.z, pf);
                            pe = fmaf(v[4 * j4 + 2], fb.z, pe);
                            pf = fmaf(v[4 * j4 + 3], fa.w, pf);
                            pe = fmaf(v[4 * j4 + 3], fb.w, pe);
                        }
                    } else {
                        // this warp's 32 columns of the NH FC2 rows, staged in its own shared
                        // slice (coalesced loads, no cross-warp wait), then read as broadcasts
                        float *myw = prm + a.w2h_off + (warp - 2) * NH * 32;
#pragma unroll
                        for (int o = 0; o < NH; o++) myw[o * 32 + lane] = __ldg(a.w2 + (size_t)o * N + col0 + lane);
                        __syncwarp();
#pragma unroll
                        for (int o = 0; o < NH; o++) {
                            const float4 *wr = reinterpret_cast<const float4 *>(myw + o * 32);
#pragma unroll
                            for (int j4 = 0; j4 < 8; j4++) {
                                const float4 w = wr[j4];
                                ph[o] = fmaf(v[4 * j4], w.x, ph[o]); ph[o] = fmaf(v[4 * j4 + 1], w.y, ph[o]);
                                ph[o] = fmaf(v[4 * j4 + 2], w.z, ph[o]); ph[o] = fmaf(v[4 * j4 + 3], w.w, ph[o]);
                            }
                        }
                        __syncwarp();   // read before the next chunk overwrites
                    }
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(stg + lane * SROW);
                    if constexpr (FP8) {
#pragma unroll
                        for (int j = 0; j < 2; j++) {
                            uint32_t w[4];
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                const int o = 16 * j + 4 * h;
                                const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[o], v[o + 1]), __NV_SATFINITE, __NV_E4M3);
                                const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[o + 2], v[o + 3]), __NV_SATFINITE, __NV_E4M3);
                                w[h] = (lo & 0xffffu) | (hi << 16);
                            }
                            dst[j] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            uint32_t w[4];
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * j + 2 * h], v[8 * j + 2 * h + 1]);
                                w[h] = *reinterpret_cast<uint32_t *>(&b2);
                            }
                            dst[j] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                    __syncwarp();
                    constexpr int U = CB / 16, RPP = 32 / U;
                    const int rr = lane / U, u = lane % U;
                    if (L.rows_plain) {   // view rows m0 + i, slot sb * 64 + i / 2
                        uint8_t *gbase = reinterpret_cast<uint8_t *>(Lt.out) + ((size_t)m0 * N + col0) * OES + u * 16;
#pragma unroll
                        for (int pass = 0; pass < U; pass++) {
                            const int r_in = pass * RPP + rr, i = q * 32 + r_in;
                            const uint4 val = *reinterpret_cast<const uint4 *>(stg + r_in * SROW + u * 16);
                            if (sb * (BM / 2) + (i >> 1) < M)
                                *reinterpret_cast<uint4 *>(gbase + (size_t)i * N * OES) = val;
                        }
                    } else {
                        // pair-major destination of output position `pos` of each slot
                        uint8_t *gbase = reinterpret_cast<uint8_t *>(Lt.out) +
                                         ((size_t)(pos >> 1) * a.B * 2 * N + (size_t)(pos & 1) * N + col0) * OES + u * 16;
#pragma unroll
                        for (int pass = 0; pass < U; pass++) {
                            const int r_in = pass * RPP + rr;
                            const int slot = m0 + q * 32 + r_in;
                            const uint4 val = *reinterpret_cast<const uint4 *>(stg + r_in * SROW + u * 16);
                            if (slot < M) *reinterpret_cast<uint4 *>(gbase + (size_t)slot * 2 * N * OES) = val;
                        }
                    }
                    __syncwarp();
                }
            }
            if (L.out_part && row < M) {
                if constexpr (NO == 2) {
                    reinterpret_cast<float2 *>(L.out)[(size_t)(2 * nt + half) * a.B + row] = make_float2(pf, pe);
                } else {
                    float *dst = reinterpret_cast<float *>(L.out) + ((size_t)(2 * nt + half) * a.B + row) * NO;
#pragma unroll
                    for (int o = 0; o < NO; o++) dst[o] = ph[o];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(acc));
        }
        if (det && warp == 2 && lane == 0) atomicAdd(&a.detail[4 * l + 2], gtimer() - t_phase);
    }
    return t_phase;
}

// The first two conv layers as one phase (plain CNN, 256 channels, k=2 / stride-2,
// Sec. 2.3).  A tile is 128 slots at one output position p of conv2; it needs conv1's
// output at positions 2p and 2p+1 of the same slots, which the tile computes itself:
// four conv1 pieces (position x 128-channel half; A from the pair-major feature rows,
// conv1's weights resident in shared memory) whose epilogues apply bias and ReLU
// (FP8: the scales) and store the values, in the layer's storage type, into tensor
// memory columns [0, 256) (BF16: two to a column; FP8: four), which is exactly
// conv2's K-major A operand [posbit * 256 + channel]; then two conv2 pieces (output
// channel halves) as MMAs with A in tensor memory and B streamed in 128-row units.
// Positions past conv1's extent read padding rows (zero features), so they come out
// as conv1's constant row, as in the unfused phases.  The six pieces of a tile use
// the two 128-column accumulators at columns 256 and 384 in turn, and each
// accumulator has its own epilogue warpgroup (warps 2-5: the first, 6-9: the
// second), so two pieces' epilogues overlap.
constexpr uint32_t kFuAcc = 256;
constexpr uint32_t kUnit = A_BYTES;   // one operand unit: 128 rows x 128 bytes
constexpr int kFuBars = 9;            // per fused phase beyond the units: 4 A quarters, weights, 2 + 2 accumulator

template <bool FP8>
__device__ uint64_t fused_phase(const PArgs &a, int l, int n2, int n2_prev, uint8_t *smem, uint64_t *bars, float *prm,
                                uint8_t *staging, uint32_t tmem_base, volatile int *cta_abort, Pipe &pp) {
    using T = typename std::conditional<FP8, __nv_fp8_e4m3, __nv_bfloat16>::type;
    const PLayer &L1 = a.layer[l], &L2 = a.layer[l + 1];
    constexpr int BK = FP8 ? 128 : 64;   // K elements per 128-byte row
    constexpr int KB1 = 128 / BK;        // conv1: K = 2 rows x 64 features
    constexpr int KB2 = 512 / BK;        // conv2: K = 2 positions x 256 channels
    constexpr int EPC = FP8 ? 4 : 2;     // A-operand elements per tensor-memory column
    const int S = a.stages, U = a.fu, F0 = kFuBar(S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t smem_base = smem_u32(smem), w1 = smem_base + (uint32_t)U * kUnit;
    auto ffull = [&](int u) { return smem_u32(&bars[F0 + u]); };
    auto fempty = [&](int u) { return smem_u32(&bars[F0 + U + u]); };
    auto a2full = [&](int i) { return smem_u32(&bars[F0 + 2 * U + i]); };
    const uint32_t w1bar = smem_u32(&bars[F0 + 2 * U + 4]);
    auto afull = [&](int x) { return smem_u32(&bars[F0 + 2 * U + 5 + x]); };
    auto aempty = [&](int x) { return smem_u32(&bars[F0 + 2 * U + 7 + x]); };
    const int M = min(*a.A->n_active, a.B);
    const int n_sb = (M + BM - 1) / BM, n_tiles = n2 * n_sb;
    const int64_t lim = a.spin_ns;
    const bool det = a.detail && blockIdx.x == 0;
    const uint64_t t_phase = det ? gtimer() : 0;
    if (a.exec && blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(&a.exec[l], (unsigned long long)(2 * n2) * (unsigned long long)M);
        atomicAdd(&a.exec[l + 1], (unsigned long long)n2 * (unsigned long long)M);
    }
    const bool any = (int)blockIdx.x < n_tiles;
    if (warp == 0) {
        if (lane == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            bool ok = true;
            if (any) {   // conv1's weights, 128-row halves of each K-block, for the phase
                mbar_expect_tx(w1bar, (uint32_t)(2 * KB1) * kUnit);
                for (int kb = 0; kb < KB1; kb++)
                    for (int h = 0; h < 2; h++)
                        tma_load_2d(w1 + (uint32_t)(kb * 2 + h) * kUnit, &a.tW1, w1bar, kb * BK, h * 128);
            }
            auto unit = [&](const CUtensorMap *m, int x, int y) {
                const int u = pp.fprod % U;
                if (!mbar_wait(fempty(u), ((uint32_t)(pp.fprod / U) & 1u) ^ 1u, lim, cta_abort, a.status)) return false;
                mbar_expect_tx(ffull(u), kUnit);
                tma_load_2d(smem_base + (uint32_t)u * kUnit, m, ffull(u), x, y);
                pp.fprod++;
                return true;
            };
            // conv1's input pairs 2p and 2p+1 of a tile's slots (pair-major rows [pair * B + slot])
            auto a1_row = [&](int t, int pb) { return (2 * (t / n_sb) + pb) * a.B + (t % n_sb) * BM; };
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                // this CTA's next tile reads its feature rows from device memory: start them into L2
                const int tn = t + (int)gridDim.x;
                if (tn < n_tiles)
                    for (int pb = 0; pb < 2; pb++)
                        for (int kb = 0; kb < KB1; kb++) tma_prefetch_2d(&L1.tA, kb * BK, a1_row(tn, pb));
                for (int pb = 0; pb < 2 && ok; pb++)
                    for (int kb = 0; kb < KB1 && ok; kb++) ok = unit(&L1.tA, kb * BK, a1_row(t, pb));
                // conv2's weights: output-channel half h, K-block kb
                for (int h = 0; h < 2 && ok; h++)
                    for (int kb = 0; kb < KB2 && ok; kb++) ok = unit(&a.tW2h, kb * BK, h * 128);
            }
        }
    } else if (warp == 1) {
        const uint32_t ID = idesc_rt(128, FP8);
        bool ok = true;
        if (any) {
            ok = __all_sync(0xffffffffu, mbar_wait(w1bar, (uint32_t)pp.fw1 & 1u, lim, cta_abort, a.status));
            pp.fw1++;
            tc_fence_after();
        }
        // CTA 0 sums the MMA warp's waits: accumulator free, operand unit, A-operand quarter
        uint64_t w_acc = 0, w_unit = 0, w_a2 = 0;
        // the next accumulator of the running piece count, once its warpgroup has drained it
        auto take = [&](uint32_t &d, int &acc) {
            acc = pp.fpc & 1;
            const uint64_t t0 = det ? gtimer() : 0;
            const bool got = __all_sync(0xffffffffu, mbar_wait(aempty(acc), ((uint32_t)(pp.fpc >> 1) & 1u) ^ 1u, lim,
                                                               cta_abort, a.status));
            if (det) w_acc += gtimer() - t0;
            if (!got) return false;
            tc_fence_after();
            d = tmem_base + kFuAcc + (uint32_t)acc * 128;
            return true;
        };
        auto wait_unit = [&](int it) {
            const uint64_t t0 = det ? gtimer() : 0;
            const bool got = __all_sync(0xffffffffu,
                                        mbar_wait(ffull(it % U), (uint32_t)(it / U) & 1u, lim, cta_abort, a.status));
            if (det) w_unit += gtimer() - t0;
            if (got) tc_fence_after();
            return got;
        };
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
            if (det && lane == 0 && t == (int)blockIdx.x) atomicAdd(&a.detail[4 * (l + 1) + 0], gtimer() - t_phase);
            // conv1: per input pair, both channel halves from the same A units
#pragma unroll
            for (int pb = 0; pb < 2; pb++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    uint32_t d;
                    int acc;
                    if (ok) ok = take(d, acc);
                    if (!ok) break;
#pragma unroll
                    for (int kb = 0; kb < KB1; kb++) {
                        const int it = pp.fmma + kb, u = it % U;
                        if (h == 0 && !(ok = wait_unit(it))) break;
                        const uint32_t a_lo = sdesc_lo(smem_base + (uint32_t)u * kUnit);
                        const uint32_t b_lo = sdesc_lo(w1 + (uint32_t)(kb * 2 + h) * kUnit);
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            umma_lo<FP8>(d, a_lo + 2u * k, b_lo + 2u * k, ID, (kb | k) != 0 ? 1u : 0u);
                        if (h == 1) umma_commit_warp(fempty(u));
                    }
                    if (!ok) break;
                    umma_commit_warp(afull(acc));
                    pp.fpc++;
                }
                if (!ok) break;
                pp.fmma += KB1;
            }
            // conv2: A = tensor-memory columns [0, 256), B = unit per K-block
#pragma unroll
            for (int h = 0; h < 2; h++) {
                uint32_t d;
                int acc;
                if (ok) ok = take(d, acc);
                if (!ok) break;
#pragma unroll
                for (int kb = 0; kb < KB2; kb++) {
                    if (h == 0 && (kb * BK) % 128 == 0) {   // this K-block's quarter of the A operand is stored
                        const uint64_t t0 = det ? gtimer() : 0;
                        ok = __all_sync(0xffffffffu, mbar_wait(a2full(kb * BK / 128), (uint32_t)pp.fz & 1u, lim,
                                                               cta_abort, a.status));
                        if (det) w_a2 += gtimer() - t0;
                        if (!ok) break;
                        tc_fence_after();
                    }
                    const int u = pp.fmma % U;
                    if (!(ok = wait_unit(pp.fmma))) break;
                    const uint32_t b_lo = sdesc_lo(smem_base + (uint32_t)u * kUnit);
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        umma_ts<FP8>(d, tmem_base + (uint32_t)(kb * 32 + k * 8), b_lo + 2u * k, ID,
                                     (kb | k) != 0 ? 1u : 0u);
                    umma_commit_warp(fempty(u));
                    pp.fmma++;
                }
                if (!ok) break;
                umma_commit_warp(afull(acc));
                pp.fpc++;
            }
            pp.fz++;
        }
        if (det && lane == 0) {
            atomicAdd(&a.detail[4 * (l + 1) + 1], gtimer() - t_phase);
            // the first layer's row (it has no phase of its own): the waits
            atomicAdd(&a.detail[4 * l + 0], w_acc);
            atomicAdd(&a.detail[4 * l + 1], w_unit);
            atomicAdd(&a.detail[4 * l + 2], w_a2);
        }
        __syncwarp();
    } else {
        fill_const<T>(a, L2, n2, n2_prev, M);   // conv2 positions this step no longer computes
        // warpgroup x = (warp - 2) / 4 drains accumulator x: the tile's pieces x, x + 2, x + 4;
        // its warp q = warp % 4 reads lanes 32q .. 32q + 31 (the hardware's lane quarters)
        const int q = warp & 3, x = (warp - 2) >> 2;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        const uint32_t src = tmem_base + lanes + kFuAcc + (uint32_t)x * 128;
        const float *b1 = prm + L1.prm_off, *s1 = b1 + L1.N;   // FP8: scale and bias folded with the
        const float *b2 = prm + L2.prm_off, *s2 = b2 + L2.N;   // requant multiplier
        constexpr int OES = FP8 ? 1 : 2;
        constexpr int CB = 32 * OES, SROW = CB + 16;
        uint8_t *stg = staging + (warp - 2) * 32 * SROW;
        // 64 accumulator columns from c0 in the storage type, lowest column in the low bits:
        // bias (FP8: dequant scale before it, both times the requant multiplier), then the ReLU,
        // which the rounding conversion applies (it commutes with round-to-nearest).
        // BF16: 32 words of two; FP8: 16 words of four.
        auto act_pack = [&](const uint32_t (&r)[64], const float *bb, const float *sc, int c0,
                            uint32_t (&w)[32]) {
            const float4 *b4 = reinterpret_cast<const float4 *>(bb + c0);
#pragma unroll
            for (int j4 = 0; j4 < 16; j4++) {
                const float4 b = b4[j4];
                float x0 = __uint_as_float(r[4 * j4]), x1 = __uint_as_float(r[4 * j4 + 1]);
                float x2 = __uint_as_float(r[4 * j4 + 2]), x3 = __uint_as_float(r[4 * j4 + 3]);
                if constexpr (FP8) {   // scale and bias carry the requant multiplier
                    const float4 s = reinterpret_cast<const float4 *>(sc + c0)[j4];
                    w[j4] = e4m3x2_relu(x0 * s.x + b.x, x1 * s.y + b.y) | (e4m3x2_relu(x2 * s.z + b.z, x3 * s.w + b.w) << 16);
                } else {
                    w[2 * j4] = bf16x2_relu(x0 + b.x, x1 + b.y);
                    w[2 * j4 + 1] = bf16x2_relu(x2 + b.z, x3 + b.w);
                }
            }
        };
        // every lane's tensor-memory accesses are complete (fence, warp sync): one arrival a warp
        auto release = [&](uint32_t bar) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar);
        };
        uint64_t w_full = 0;   // CTA 0, warp 2: waits for a full accumulator
        auto wait_full = [&]() {
            const uint64_t t0 = det ? gtimer() : 0;
            const bool got = __all_sync(0xffffffffu,
                                        mbar_wait(afull(x), (uint32_t)pp.fe & 1u, lim, cta_abort, a.status));
            if (det) w_full += gtimer() - t0;
            pp.fe++;
            if (got) tc_fence_after();
            return got;
        };
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const int p2 = t / n_sb, sb = t % n_sb;
            bool ok = true;
            // conv1 pieces i = x, x + 2: position pb = i / 2, channel half h = x, in two 64-column
            // chunks, each to its A-operand columns
            for (int pb = 0; pb < 2 && ok; pb++) {
                if (!(ok = wait_full())) break;
#pragma unroll 1
                for (int c = 0; c < 2; c++) {
                    const int ch = x * 128 + c * 64;
                    uint32_t r[64], w[32];
                    tmem_ld64(src + (uint32_t)(c * 64), r);
                    if (c == 1) release(aempty(x));   // the accumulator is in registers
                    act_pack(r, b1, s1, ch, w);
                    const uint32_t dst = tmem_base + lanes + (uint32_t)((pb * 256 + ch) / EPC);
                    if constexpr (FP8) tmem_st16(dst, *reinterpret_cast<const uint32_t(*)[16]>(w));
                    else tmem_st32(dst, w);
                }
                tmem_st_wait();
                release(a2full(2 * pb + x));
            }
            if (!ok) break;
            // conv2 piece 4 + x: output channels x * 128 + [0, 128) of position p2, two 64-column
            // chunks, each in two 32-column halves through the warp's staging rows to the
            // pair-major destination of position p2 of each slot (16-byte pieces in row passes)
            if (!(ok = wait_full())) break;
#pragma unroll 1
            for (int c = 0; c < 2; c++) {
                const int ch = x * 128 + c * 64;
                uint32_t r[64], w[32];
                tmem_ld64(src + (uint32_t)(c * 64), r);
                if (c == 1) release(aempty(x));   // the accumulator is in registers
                act_pack(r, b2, s2, ch, w);
                constexpr int WPH = 32 / EPC;   // words per 32-column half
                constexpr int UU = CB / 16, RPP = 32 / UU;
                const int rr = lane / UU, uu = lane % UU;
#pragma unroll
                for (int hf = 0; hf < 2; hf++) {
                    uint4 *dst = reinterpret_cast<uint4 *>(stg + lane * SROW);
#pragma unroll
                    for (int j = 0; j < WPH / 4; j++)
                        dst[j] = make_uint4(w[hf * WPH + 4 * j], w[hf * WPH + 4 * j + 1], w[hf * WPH + 4 * j + 2],
                                            w[hf * WPH + 4 * j + 3]);
                    __syncwarp();
                    uint8_t *gbase = reinterpret_cast<uint8_t *>(L2.out) +
                                     ((size_t)(p2 >> 1) * a.B * 2 * L2.N + (size_t)(p2 & 1) * L2.N + ch + 32 * hf) * OES +
                                     uu * 16;
#pragma unroll
                    for (int pass = 0; pass < UU; pass++) {
                        const int r_in = pass * RPP + rr;
                        const int slot = sb * BM + q * 32 + r_in;
                        const uint4 val = *reinterpret_cast<const uint4 *>(stg + r_in * SROW + uu * 16);
                        if (slot < M) *reinterpret_cast<uint4 *>(gbase + (size_t)slot * 2 * L2.N * OES) = val;
                    }
                    __syncwarp();
                }
            }
        }
        if (det && warp == 2 && lane == 0) {
            atomicAdd(&a.detail[4 * (l + 1) + 2], gtimer() - t_phase);
            atomicAdd(&a.detail[4 * l + 3], w_full);
        }
    }
    return t_phase;
}

template <bool FP8, int NO>
__global__ void __launch_bounds__(kThreads, 1) persist_kernel(const __grid_constant__ PArgs a) {
    using T = typename std::conditional<FP8, __nv_fp8_e4m3, __nv_bfloat16>::type;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int S = a.stages;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + a.ring_bytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 4);
    volatile int *cta_abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *prm = reinterpret_cast<float *>(smem + a.ring_bytes + kBarBytes);
    uint8_t *staging = reinterpret_cast<uint8_t *>(prm + a.prm_floats);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[S + s]), 1);
        }
        for (int x = 0; x < 2; x++) {
            mbar_init(smem_u32(&bars[2 * S + x]), 1);
            mbar_init(smem_u32(&bars[2 * S + 2 + x]), kEpiWarps);   // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&bars[2 * S + 5]), 1);   // resident weights (after tmem_slot and cta_abort)
        if (a.fuse) {
            const int F0 = kFuBar(S);
            for (int u = 0; u < a.fu; u++) {
                mbar_init(smem_u32(&bars[F0 + u]), 1);
                mbar_init(smem_u32(&bars[F0 + a.fu + u]), 1);
            }
            // A-operand quarters and accumulator-free barriers: one arrival per warp of a warpgroup
            for (int i = 0; i < 4; i++) mbar_init(smem_u32(&bars[F0 + 2 * a.fu + i]), kEpiWarps / 2);
            mbar_init(smem_u32(&bars[F0 + 2 * a.fu + 4]), 1);
            for (int x = 0; x < 2; x++) {
                mbar_init(smem_u32(&bars[F0 + 2 * a.fu + 5 + x]), 1);
                mbar_init(smem_u32(&bars[F0 + 2 * a.fu + 7 + x]), kEpiWarps / 2);
            }
        }
        *cta_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    unsigned target = 0;
    Pipe pp;
    uint64_t t_prev = gtimer();
    auto mark = [&](int kind) {  // CTA 0 attributes the time since the last barrier to `kind`
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.phase_ns) {
            const uint64_t t = gtimer();
            a.phase_ns[kind] += t - t_prev;
            a.phase_n[kind] += 1;
            t_prev = t;
        }
    };
    // every layer's parameters, once for the call
    for (int l = 0; l < a.n_layers; l++) {
        const PLayer &L = a.layer[l];
        float *pb = prm + L.prm_off;
        const int N = L.N;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            pb[i] = L.bias[i];
            if (FP8) {
                // a conv layer's requant multiplier o (> 0) is folded in: max(x s + b, 0) o =
                // max(x (s o) + b o, 0), one FMA before the saturating conversion
                const float o = L.oscale ? L.oscale[i] : 1.f;
                const bool fold = !L.out_part && L.relu;
                pb[N + i] = fold ? L.scale[i] * o : L.scale[i];
                pb[2 * N + i] = o;
                if (fold) pb[i] = L.bias[i] * o;
            }
            if (NO == 2 && L.out_part) {   // the hybrid / store heads stage their FC2 rows per warp
                float *w = pb + (FP8 ? 3 * N : N);
                w[i] = a.w2[i];
                w[N + i] = a.w2[N + i];
            }
        }
    }
    __syncthreads();
    gather_phase<T>(a, smem, a.ext);
    bool ok = grid_sync(a, target, cta_abort);
    mark(SIMNET_KERNEL_GATHER);
    // positions per layer for a batch extent x (rows in use: the longest context + 1)
    auto layer_pos = [&](const PLayer &L, int x) {
        return max(1, min(L.rows_out, (x + (1 << L.pos_log) - 1) >> L.pos_log));
    };
    int ext_prev = a.A->window;   // tiles hold stale rows at the start: fill every position
    for (int64_t step = 0; step < a.n_steps && ok; step++) {
        int *ext_now = a.ext + (step & 1), *ext_next = a.ext + ((step + 1) & 1);
        const int ext = *(volatile int *)ext_now;
        int e = (ext + (1 << a.n_conv) - 1) >> a.n_conv;  // last conv-output rows
        e = (e + a.e_round - 1) / a.e_round * a.e_round;
        e = max(1, min(e, a.rows_n));
        if (blockIdx.x == 0 && threadIdx.x == 0) *ext_next = 0;   // the head phase raises it
        int ph = 0;   // GEMM phases of this step so far (odd ones walk their tiles backwards)
        for (int l = 0; l < a.n_layers && ok; l++, ph++) {
            const PLayer &L = a.layer[l];
            if (l == 0 && a.fuse) {   // conv1 and conv2 in one phase
                const int n2 = layer_pos(a.layer[1], ext), n2_prev = layer_pos(a.layer[1], ext_prev);
                const uint64_t tp = fused_phase<FP8>(a, 0, n2, n2_prev, smem, bars, prm, staging, tmem_base, cta_abort, pp);
                l = 1;
                ok = grid_sync(a, target, cta_abort);
                if (a.detail && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.detail[4 * l + 3], gtimer() - tp);
                mark(SIMNET_KERNEL_LAYER0 + a.layer[l].kind);
                continue;
            }
            const int n_now = L.out_part ? 1 : layer_pos(L, ext), n_prev = L.out_part ? 1 : layer_pos(L, ext_prev);
            const int l2 = L.pair_next ? l + 1 : -1;   // a residual block's conv takes its projection along
            const uint64_t tp =
                gemm_phase<FP8, NO>(a, l, l2, e, n_now, n_prev, smem, bars, prm, staging, tmem_base, cta_abort, pp,
                                    (ph & 1) != 0);
            if (l2 >= 0) l++;
            ok = grid_sync(a, target, cta_abort);
            if (a.detail && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.detail[4 * l + 3], gtimer() - tp);
            mark(SIMNET_KERNEL_LAYER0 + a.layer[l].kind);
        }
        if (!ok) break;
        ext_prev = ext;
        {   // head phase: every warp of the grid takes slots; the stage ring is its scratch.
            // Software-pipelined over a warp's slots: the sub-trace of the slot two ahead and
            // the state and FC2 partials of the next one are loaded before this one is
            // processed, so their device-memory round trips overlap its work.
            constexpr int PER = 256 * 8 + 32 * stage_row_bytes<T>();
            uint8_t *mine = smem + warp * PER;
            const int n_act = *a.A->n_active, stride = gridDim.x * kWarps;
            int slot = blockIdx.x * kWarps + warp;
            HeadState cur;
            int ext_run = 0;   // this warp's largest next-step extent, published once (one atomic
                               // per warp: an atomic per slot on one address serialises in L2)
            if (slot < n_act) head_load<NO>(a.A, slot, a.A->active[slot], lane, a.part, a.P, a.B, cur);
            int b_next = slot + stride < n_act ? a.A->active[slot + stride] : 0;
            for (; slot < n_act; slot += stride) {
                const int s1 = slot + stride, s2 = slot + 2 * stride;
                const int b_after = s2 < n_act ? a.A->active[s2] : 0;
                HeadState nxt;
                if (s1 < n_act) head_load<NO>(a.A, s1, b_next, lane, a.part, a.P, a.B, nxt);
                head_update_state<T, NO>(a.A, slot, lane, cur, a.part, a.P, a.B, a.b2, reinterpret_cast<T *>(a.X),
                                         reinterpret_cast<uint64_t *>(mine), mine + 256 * 8, a.B, &ext_run);
                cur = nxt;
                b_next = b_after;
            }
            if (lane == 0 && ext_run > 0) atomicMax(ext_next, ext_run);
        }
        ok = grid_sync(a, target, cta_abort);
        mark(SIMNET_KERNEL_HEAD_UPDATE);
        if (ok && a.compact_every > 0 && (step + 1) % a.compact_every == 0 && step + 1 < a.n_steps) {
            if (blockIdx.x == 0) compact_block(a.A);
            ok = grid_sync(a, target, cta_abort);
            mark(SIMNET_KERNEL_COMPACT);
            if (!ok) break;
            gather_phase<T>(a, smem, ext_next);
            ok = grid_sync(a, target, cta_abort);
            mark(SIMNET_KERNEL_GATHER);
            ext_prev = a.A->window;   // slots moved: every tile position is stale
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
}

}  // namespace

// Host side: fill the argument block from the layer plans and launch.
bool launch_persistent(simnet_ctx *c, int B, int64_t n_steps, bool uneven, cudaStream_t s, std::string &why) {
    PArgs a;
    memset(&a, 0, sizeof a);
    const bool fp8 = c->cfg.precision == SIMNET_FP8_E4M3;
    int bn_max = 64, n_max = 0;
    const int BK = fp8 ? 128 : 64;
    const int C = c->cfg.conv_channels, W = c->cfg.window;
    // every conv-stack layer writes its own pair-major tile (the per-layer extent keeps
    // constant rows in it past the extent, so tiles cannot be shared between layers)
    const size_t es = fp8 ? 1 : 2;
    if (c->pbuf_B < B) {
        for (auto &q : c->pbuf)
            if (q) { cudaFree(q); q = nullptr; }
        c->pbuf_B = 0;
        for (int l = 0; l + 1 < c->n_layers; l++) {
            const int blk = c->residual ? l / 3 : l, rows_out = W >> (blk + 1);
            const size_t bytes = (size_t)B * (2 * ((rows_out + 1) / 2)) * C * es;
            if (cudaMalloc(&c->pbuf[l], bytes) != cudaSuccess) { why = "out of memory for layer tiles"; return false; }
        }
        c->pbuf_B = B;
    }
    // the layer that last wrote each workspace buffer id (inputs follow the producers)
    int writer[6] = {-1, -1, -1, -1, -1, -1};
    for (int l = 0; l < c->n_layers; l++) {
        const TcPlan &p = c->plan[l];
        const GemmLayer &g = c->layer[l];
        PLayer &L = a.layer[l];
        const bool fc1 = l == c->n_layers - 1;
        const int blk = fc1 ? c->cfg.n_conv : c->residual ? l / 3 : l;   // conv layer / residual block
        const bool pw = c->residual && !fc1 && l % 3 == 2;
        const void *in = g.in_buf == kBufX ? c->X : c->pbuf[writer[g.in_buf]];
        if (pw) {
            // positions of the block output viewed as [2 * pairs * B][C]
            const int rows_out = W >> (blk + 1);
            if (!encode_map_2d(L.tA, c->cfg.precision, in, (uint64_t)C, (uint64_t)2 * ((rows_out + 1) / 2) * B, BK,
                               BM, why))
                return false;
        } else {
            // input rows of this layer and its pair-major view [pairs * B][2 * row width]
            const int in_rows = W >> blk;
            const int row_w = blk == 0 ? kNFP : C;
            if (!encode_map_2d(L.tA, c->cfg.precision, in, (uint64_t)2 * row_w, (uint64_t)((in_rows + 1) / 2) * B, BK,
                               BM, why))
                return false;
        }
        L.tB = p.tB;
        L.bias = g.bias;
        L.scale = g.scale;
        L.oscale = g.oscale;
        L.out = fc1 ? (void *)c->h1 : c->pbuf[l];
        L.K = g.K;
        L.N = g.N;
        L.BN = p.BN;
        L.out_part = fc1;
        L.n_tiles_n = g.N / p.BN;
        L.cin = blk == 0 ? kNFP : C;
        L.pos_shift = fc1 ? 0 : c->cfg.n_conv - 1 - blk;
        L.relu = g.relu;
        L.rows_plain = pw;
        L.resid = g.res_buf >= 0 ? c->pbuf[writer[g.res_buf]] : nullptr;
        L.kind = g.kind;
        L.pos_log = blk + 1;
        L.pair_next = c->residual && !fc1 && l % 3 == 0;
        L.rows_out = fc1 ? 1 : W >> (blk + 1);
        L.cst = fc1 ? nullptr : c->layer_const + (size_t)l * C;
        if (!fc1) writer[g.out_buf] = l;
        bn_max = std::max(bn_max, p.BN);
        n_max = std::max(n_max, g.N);
    }
    a.n_conv = c->cfg.n_conv;
    a.fc1_const = c->fc1_const;
    a.ext = c->ext;
    a.rows_n = c->rows_n;
    a.e_round = std::max(1, BK / C);
    a.A = c->d_args;
    a.X = c->X;
    a.part = c->h1;
    a.w2 = c->w2;
    a.b2 = c->b2;
    a.bar_counter = c->bar;
    a.abort_g = c->bar_abort;
    a.status = c->status;
    a.phase_ns = c->phase_on ? c->phase_ns : nullptr;
    a.phase_n = c->phase_on ? c->phase_n : nullptr;
    // per-GEMM detail has room for the layers of a plain CNN (4 counters each)
    a.detail = c->phase_on && c->n_layers <= kMaxConv + 1 ? c->phase_ns + 16 : nullptr;
    a.exec = c->phase_on && c->n_layers <= 8 ? c->phase_ns + 40 : nullptr;
    a.n_steps = n_steps;
    a.spin_ns = c->cfg.spin_limit_ns;
    a.bar_spin_ns = c->cfg.barrier_limit_us > 0 ? (int64_t)c->cfg.barrier_limit_us * 1000 : c->cfg.spin_limit_ns;
    a.n_layers = c->n_layers;
    a.B = B;
    a.P = c->n_part;
    a.compact_every = uneven ? 16 : 0;
    a.stage_bytes = A_BYTES + bn_max * ROW_BYTES;
    // shared parameter table: per layer bias (+ FP8 scale, requant) (+ FC1's FC2 rows),
    // then FC1's per-step padding row, then the per-warp FC2 row slices of wider heads
    int off = 0;
    for (int l = 0; l < c->n_layers; l++) {
        a.layer[l].prm_off = off;
        const int N = a.layer[l].N;
        off += N * (fp8 ? 3 : 1) + (a.layer[l].out_part && c->n_out == 2 ? 2 * N : 0);
        off = (off + 3) & ~3;   // 16-byte aligned blocks
    }
    a.cst_off = off;
    off += a.layer[c->n_layers - 1].N;
    a.w2h_off = (off + 3) & ~3;
    a.prm_floats = a.w2h_off + (c->n_out == 2 ? 0 : kEpiWarps * c->n_out * 32);
    const size_t staging = (size_t)kEpiWarps * 32 * (32 * (fp8 ? 1 : 2) + 16);
    const size_t fixed = 1024 + kBarBytes + (size_t)a.prm_floats * 4 + staging;
    const size_t budget = 232448 - 1024;   // minus the static shared memory of the compaction
    a.stages = (int)std::min<size_t>(6, (budget - fixed) / a.stage_bytes);
    // the head phase reuses the stage ring as 10 x 256 queue entries: fewest stages that hold them
    const size_t head_scratch = (size_t)kWarps * (256 * 8 + 32 * (kNFP * 4 + 16));
    const int min_stages = std::max<int>(2, (int)((head_scratch + a.stage_bytes - 1) / a.stage_bytes));
    if (c->tuned_B == B && c->tuned_persist_stages >= 2 && c->tuned_persist_stages < a.stages)
        a.stages = std::max(c->tuned_persist_stages, min_stages);   // the autotuner's pick
    if (a.stages < 2) { why = "shared memory budget"; return false; }
    if ((size_t)a.stages * a.stage_bytes < head_scratch) {
        why = "ring too small for the head and gather scratch";
        return false;
    }
    // conv1 + conv2 in one phase: conv1's weights stay in shared memory for the phase,
    // and 16 KB operand units fill the room left (the ring and the shared memory the
    // stages leave unused)
    a.fuse = 0;
    if (!(c->cfg.flags & SIMNET_FLAG_NO_FUSE) && !c->residual && c->cfg.n_conv >= 2 && C == 256 &&
        c->layer[0].K == 2 * kNFP && c->layer[0].N == C && c->layer[1].K == 2 * C && c->layer[1].N == C &&
        c->n_layers > 2) {
        const int w1_units = 2 * (2 * kNFP * (int)es / ROW_BYTES);
        // as many units as the shared memory left beside the fixed part holds, within the barrier area
        const int room = (int)((budget - fixed) / A_BYTES), cap = (kBarBytes / 8 - kFuBar(a.stages) - kFuBars) / 2;
        const int U = std::min(cap, room - w1_units);
        if (U >= 3) {
            if (!encode_map_2d(a.tW1, c->cfg.precision, c->layer[0].B, (uint64_t)c->layer[0].K, (uint64_t)C, BK, 128,
                               why) ||
                !encode_map_2d(a.tW2h, c->cfg.precision, c->layer[1].B, (uint64_t)c->layer[1].K, (uint64_t)C, BK, 128,
                               why))
                return false;
            a.fuse = 1;
            a.fu = U;
        }
    }
    a.ring_bytes = std::max(a.stages * a.stage_bytes, a.fuse ? (a.fu + 2 * (int)es) * A_BYTES : 0);
    const size_t smem = (size_t)a.ring_bytes + fixed;
    void (*k)(PArgs) = nullptr;
    switch (c->n_out) {
        case 3: k = fp8 ? persist_kernel<true, 3> : persist_kernel<false, 3>; break;
        case 22: k = fp8 ? persist_kernel<true, 22> : persist_kernel<false, 22>; break;
        case 33: k = fp8 ? persist_kernel<true, 33> : persist_kernel<false, 33>; break;
        default: k = fp8 ? persist_kernel<true, 2> : persist_kernel<false, 2>; break;
    }
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
    if (per_sm < 1) { why = "persistent kernel does not fit on an SM"; return false; }
    cudaMemsetAsync(c->bar, 0, sizeof(unsigned), s);
    cudaMemsetAsync(c->ext, 0, 2 * sizeof(int), s);
    cudaMemsetAsync(c->bar_abort, 0, sizeof(int), s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(num_sms());
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return false; }
    return true;
}

}  // namespace simnet
