// train_tc.cu -- the GEMMs of the BF16 training step (Sec. 2.4) on tcgen05
// tensor cores.
//
// A training step needs, per layer, three products over the same contiguous
// reshapes the forward uses (a k=2 / stride-2 convolution is a GEMM over row
// pairs): the forward Y = ReLU(A W^T + b), the input gradient
// dA = (dY W) * [A > 0] and the weight gradient dW = dY^T A.  They differ in
// which dimension of each stored operand is the reduction:
//   forward     A [M][K] reduces over its contiguous K        (K-major A and B)
//   input grad  dY [M][N] reduces over N (K-major), W [N][K] reduces over its
//               rows, with K contiguous                       (MN-major B)
//   weight grad A [M][K] and dY [M][N] both reduce over their rows M
//               (both MN-major), M split over the CTAs and summed atomically
// tcgen05 reads either layout straight from shared memory (the transpose bits
// of the instruction descriptor), so no operand is ever transposed in memory.
//
// Persistent, warp-specialised kernel, one CTA per SM (the structure of the
// inference GEMM): warp 0 issues TMA loads (128-byte swizzle) into an S-stage
// ring, warp 1's elected thread issues tcgen05.mma (M = 128, N = BN, K = 16,
// FP32 accumulators in TMEM, two of them so that one tile's epilogue overlaps
// the next tile's MMAs), warps 2-9 run the epilogue from tcgen05.ld.  Every
// wait is bounded; an expired wait records a timeout in the status word, the
// CTA lets its own copies in flight land, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"
#include "train_tc.cuh"

namespace simnet {
namespace {

using namespace tcx;

constexpr int kAtomBytes = 64 * ROW_BYTES;   // one 64-row x 128-byte swizzled box (MN-major operand piece)

struct TgArgs {
    const float *bias;
    const __nv_bfloat16 *mask;
    void *out;
    float *part;   // split partial tiles [splits][N][ldo], or null
    int M, N, R, ldo;
    int n_tiles_n, m_tiles, splits, kb_per_split;
    int64_t spin_ns;
    int32_t *status;
};

// Shared-memory descriptor of an MN-major operand piece: 64-element (128-byte)
// rows along MN, one row per reduction index, 128-byte swizzle; 8-row groups
// along the reduction 1024 bytes apart (stride byte offset) and consecutive
// 64-element MN chunks one box (8 KB) apart (leading byte offset).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kAtomBytes >> 4) << 16;   // leading byte offset: next 64 MN elements
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8 reduction rows
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, M = 128, N = BN; bit 15 / 16
// select an MN-major A / B.
template <int BN, bool AMN, bool BMN>
__device__ __forceinline__ constexpr uint32_t tg_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((AMN ? 1u : 0u) << 15) | ((BMN ? 1u : 0u) << 16) |
           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int BN, int STAGES>
struct TgLayout {
    static constexpr int B_BYTES = BN * ROW_BYTES;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int RING = STAGES * STAGE_BYTES;
    static constexpr int BARS = (2 * STAGES + 5) * 8 + 16;
    static constexpr int EPI_WARPS = 8;
};

// Work item t: (reduction split, row tile, column tile) -> first row, column
// tile index and the range of 64-wide reduction blocks.
__device__ __forceinline__ void tg_decode(const TgArgs &a, int t, int &m0, int &nt, int &kb0, int &kb1,
                                          int *split_out = nullptr) {
    const int per_split = a.m_tiles * a.n_tiles_n;
    const int split = t / per_split, rem = t % per_split;
    if (split_out) *split_out = split;
    m0 = (rem / a.n_tiles_n) * BM;
    nt = rem % a.n_tiles_n;
    kb0 = split * a.kb_per_split;
    kb1 = min((a.R + 63) / 64, kb0 + a.kb_per_split);
}

template <int BN, int STAGES, bool AMN, bool BMN, int EPI>
__global__ void __launch_bounds__(320, 1)
    tg_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const TgArgs a) {
    using L = TgLayout<BN, STAGES>;
    constexpr uint32_t TMEM_COLS = 2 * BN;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::RING);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t smem_base = smem_u32(smem);
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto tfull = [&](int x) { return smem_u32(&bars[2 * STAGES + x]); };
    auto tempty = [&](int x) { return smem_u32(&bars[2 * STAGES + 2 + x]); };
    const uint32_t fin = smem_u32(&bars[2 * STAGES + 4]);   // every MMA of the CTA done

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int x = 0; x < 2; x++) {
            mbar_init(tfull(x), 1);
            mbar_init(tempty(x), 32 * L::EPI_WARPS);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tB)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int items = a.m_tiles * a.n_tiles_n * a.splits;
    const int64_t lim = a.spin_ns;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < items && ok; t += gridDim.x) {
                int m0, nt, kb0, kb1;
                tg_decode(a, t, m0, nt, kb0, kb1);
                const int n0 = nt * BN;
                for (int kb = kb0; kb < kb1; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(empty(s), ph ^ 1u, lim, abort_flag, a.status)) { ok = false; break; }
                    const uint32_t sa = smem_base + s * L::STAGE_BYTES, sb = sa + A_BYTES;
                    const int r0 = kb * 64;
                    mbar_expect_tx(full(s), L::STAGE_BYTES);
                    if constexpr (AMN) {
                        tma_load_2d(sa, &tA, full(s), m0, r0);
                        tma_load_2d(sa + kAtomBytes, &tA, full(s), m0 + 64, r0);
                    } else {
                        tma_load_2d(sa, &tA, full(s), r0, m0);
                    }
                    if constexpr (BMN) {
#pragma unroll
                        for (int j = 0; j < BN / 64; j++) tma_load_2d(sb + j * kAtomBytes, &tB, full(s), n0 + 64 * j, r0);
                    } else {
                        tma_load_2d(sb, &tB, full(s), r0, n0);
                    }
                }
            }
            if (!ok) {   // the copies already issued land before the CTA's memory is released
                for (int j = max(0, it - STAGES); j < it; j++) {
                    volatile int never = 0;
                    mbar_wait(full(j % STAGES), (uint32_t)(j / STAGES) & 1u, lim, &never, a.status);
                }
            }
        }
    } else if (warp == 1) {
        {   // the whole warp runs the issue loop, one elected lane issues (umma_warp)
            int it = 0, tc = 0;
            bool ok = true;
            constexpr uint32_t ID = tg_idesc<BN, AMN, BMN>();
            for (int t = blockIdx.x; t < items && ok; t += gridDim.x, tc++) {
                int m0, nt, kb0, kb1;
                tg_decode(a, t, m0, nt, kb0, kb1);
                const int acc = tc & 1;
                const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait(tempty(acc), aph ^ 1u, lim, abort_flag, a.status))) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int kb = kb0; kb < kb1; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!__all_sync(0xffffffffu, mbar_wait(full(s), ph, lim, abort_flag, a.status))) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_base + s * L::STAGE_BYTES, sb = sa + A_BYTES;
                    const uint64_t ad = AMN ? sdesc_mn(sa) : sdesc(sa);
                    const uint64_t bd = BMN ? sdesc_mn(sb) : sdesc(sb);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        // K = 16 per MMA: 32 bytes along a K-major row, or 16 rows (2 KB) of an
                        // MN-major piece
                        const uint64_t ak = ad + (uint64_t)(AMN ? k * 128 : k * 2);
                        const uint64_t bk = bd + (uint64_t)(BMN ? k * 128 : k * 2);
                        umma_warp<false>(d, ak, bk, ID, (kb != kb0 || k != 0) ? 1u : 0u);
                    }
                    umma_commit_warp(empty(s));
                }
                if (ok) umma_commit_warp(tfull(acc));
            }
            // MMAs still in flight after an abort finish before TMEM is released
            umma_commit_warp(fin);
            volatile int never = 0;
            mbar_wait(fin, 0u, lim > 200000000 ? lim : 200000000, &never, a.status);
        }
        __syncwarp();
    } else {
        // epilogue, warps 2..9: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows) and the
        // column half (w - 2) / 4 of the tile
        const int q = warp & 3, half = (warp - 2) >> 2;
        int tc = 0;
        for (int t = blockIdx.x; t < items; t += gridDim.x, tc++) {
            int m0, nt, kb0, kb1, split;
            tg_decode(a, t, m0, nt, kb0, kb1, &split);
            const int n0 = nt * BN;
            const int acc = tc & 1;
            const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
            const int m = m0 + q * 32 + lane;
            const bool valid = m < a.M;
            // DGRAD: this row's mask one chunk ahead; the first chunk's is loaded while
            // the tile's MMAs still run
            uint4 mk_next[4];
            if constexpr (EPI == TG_DGRAD) {
                if (valid) {
                    const uint4 *mk = reinterpret_cast<const uint4 *>(a.mask + (size_t)m * a.N + n0 + half * (BN / 2));
#pragma unroll
                    for (int j = 0; j < 4; j++) mk_next[j] = mk[j];
                }
            }
            if (!mbar_wait(tfull(acc), aph, lim, abort_flag, a.status)) break;
            tc_fence_after();
#pragma unroll 1
            for (int ch = 0; ch < BN / 64; ch++) {
                const int c = half * (BN / 2) + ch * 32;   // tile column of this chunk
                uint4 mkv[4];
                if constexpr (EPI == TG_DGRAD) {
#pragma unroll
                    for (int j = 0; j < 4; j++) mkv[j] = mk_next[j];
                    if (valid && ch + 1 < BN / 64) {
                        const uint4 *mk = reinterpret_cast<const uint4 *>(a.mask + (size_t)m * a.N + n0 + c + 32);
#pragma unroll
                        for (int j = 0; j < 4; j++) mk_next[j] = mk[j];
                    }
                }
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c), r);
                const int n = n0 + c;
                if constexpr (EPI == TG_FWD_F32) {
                    if (a.part) {   // a split reduction: this split's raw sums (bias, ReLU after the sum)
                        if (valid) {
                            float4 *o = reinterpret_cast<float4 *>(a.part + ((size_t)split * a.M + m) * a.N + n);
#pragma unroll
                            for (int j = 0; j < 8; j++)
                                o[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                                   __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                        }
                        continue;
                    }
                }
                if constexpr (EPI == TG_FWD_BF16 || EPI == TG_FWD_F32) {
                    float v[32];
                    const float4 *b4 = reinterpret_cast<const float4 *>(a.bias + n);
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const float4 b = b4[j];
                        v[4 * j] = fmaxf(__uint_as_float(r[4 * j]) + b.x, 0.f);
                        v[4 * j + 1] = fmaxf(__uint_as_float(r[4 * j + 1]) + b.y, 0.f);
                        v[4 * j + 2] = fmaxf(__uint_as_float(r[4 * j + 2]) + b.z, 0.f);
                        v[4 * j + 3] = fmaxf(__uint_as_float(r[4 * j + 3]) + b.w, 0.f);
                    }
                    if (valid) {
                        if constexpr (EPI == TG_FWD_BF16) {
                            uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(a.out) +
                                                                 (size_t)m * a.N + n);
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                uint32_t w[4];
#pragma unroll
                                for (int u = 0; u < 4; u++) {
                                    __nv_bfloat162 p = __floats2bfloat162_rn(v[8 * j + 2 * u], v[8 * j + 2 * u + 1]);
                                    w[u] = *reinterpret_cast<uint32_t *>(&p);
                                }
                                o[j] = make_uint4(w[0], w[1], w[2], w[3]);
                            }
                        } else {
                            float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + (size_t)m * a.N + n);
#pragma unroll
                            for (int j = 0; j < 8; j++) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        }
                    }
                } else if constexpr (EPI == TG_DGRAD) {
                    if (valid) {
                        uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(a.out) + (size_t)m * a.N + n);
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const uint4 mv = mkv[j];
                            const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
                            uint32_t w[4];
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                const __nv_bfloat162 y = *reinterpret_cast<const __nv_bfloat162 *>(&mw[u]);
                                const float lo = __bfloat162float(y.x) > 0.f ? __uint_as_float(r[8 * j + 2 * u]) : 0.f;
                                const float hi = __bfloat162float(y.y) > 0.f ? __uint_as_float(r[8 * j + 2 * u + 1]) : 0.f;
                                __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
                                w[u] = *reinterpret_cast<uint32_t *>(&p);
                            }
                            o[j] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                } else {   // TG_WGRAD: out[n][m] = C[m][n]; a warp's 32 rows are consecutive in memory
                    if (valid) {
                        float *dst = a.part ? a.part + (size_t)split * a.N * a.ldo : reinterpret_cast<float *>(a.out);
                        float *o = dst + (size_t)n * a.ldo + m;
#pragma unroll
                        for (int j = 0; j < 32; j++) o[(size_t)j * a.ldo] = __uint_as_float(r[j]);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty(acc));
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
    }
}

template <int BN> constexpr int tg_stages() { return BN == 256 ? 4 : BN == 128 ? 6 : 8; }

// out[i] = sum over s of part[s][i], then (forward) + bias[i % N] and ReLU: the
// splits of a reduction, summed in a fixed order.  A block takes 32 consecutive
// elements; its 8 warps sum every 8th split each, then one warp adds the 8.
// The same four columns at a time (count a multiple of 4): 16-byte loads, a block
// covers 128 consecutive outputs.
__global__ void __launch_bounds__(256) tg_reduce4_kernel(const float *__restrict__ part, int splits, int64_t count,
                                                         float *__restrict__ out, const float *__restrict__ bias, int N,
                                                         int relu) {
    __shared__ float4 sh[8][32];
    const int e = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t i4 = (int64_t)blockIdx.x * 32 + e, c4 = count / 4;
    const float4 *p4 = reinterpret_cast<const float4 *>(part);
    auto add = [](float4 &a, const float4 &b) {
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    };
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i4 < c4) {   // four independent loads in flight per thread
        float4 s1 = s, s2 = s, s3 = s;
        int k = g;
        for (; k + 24 < splits; k += 32) {
            add(s, p4[(size_t)k * c4 + i4]);
            add(s1, p4[(size_t)(k + 8) * c4 + i4]);
            add(s2, p4[(size_t)(k + 16) * c4 + i4]);
            add(s3, p4[(size_t)(k + 24) * c4 + i4]);
        }
        for (; k < splits; k += 8) add(s, p4[(size_t)k * c4 + i4]);
        add(s, s1);
        add(s2, s3);
        add(s, s2);
    }
    sh[g][e] = s;
    __syncthreads();
    if (g == 0 && i4 < c4) {
        float4 t = sh[0][e];
#pragma unroll
        for (int q = 1; q < 8; q++) add(t, sh[q][e]);
        float v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (bias) v[j] += bias[(4 * i4 + j) % N];
            if (relu) v[j] = fmaxf(v[j], 0.f);
        }
        reinterpret_cast<float4 *>(out)[i4] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

__global__ void __launch_bounds__(256) tg_reduce_kernel(const float *__restrict__ part, int splits, int64_t count,
                                                        float *__restrict__ out, const float *__restrict__ bias, int N,
                                                        int relu) {
    __shared__ float sh[8][33];
    const int e = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + e;
    float s = 0.f;
    if (i < count) {   // four independent loads in flight per thread
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int k = g;
        for (; k + 24 < splits; k += 32) {
            s0 += part[(size_t)k * count + i];
            s1 += part[(size_t)(k + 8) * count + i];
            s2 += part[(size_t)(k + 16) * count + i];
            s3 += part[(size_t)(k + 24) * count + i];
        }
        for (; k < splits; k += 8) s0 += part[(size_t)k * count + i];
        s = (s0 + s1) + (s2 + s3);
    }
    sh[g][e] = s;
    __syncthreads();
    if (g == 0 && i < count) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; q++) t += sh[q][e];
        if (bias) t += bias[i % N];
        if (relu) t = fmaxf(t, 0.f);
        out[i] = t;
    }
}

template <int BN, bool AMN, bool BMN, int EPI>
void tg_launch_one(const TgPlan &p, const TgArgs &a, cudaStream_t s) {
    constexpr int ST = tg_stages<BN>();
    auto k = tg_kernel<BN, ST, AMN, BMN, EPI>;
    static size_t attr = 0;
    if (attr < p.smem) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        attr = p.smem;
    }
    k<<<p.grid, 320, p.smem, s>>>(p.tA, p.tB, a);
}

template <int BN, int EPI>
void tg_launch_bn(const TgPlan &p, const TgArgs &a, cudaStream_t s) {
    // the layouts the training step uses: forward (K, K), input gradient (K, MN),
    // weight gradient (MN, MN)
    if (!p.a_mn && !p.b_mn) tg_launch_one<BN, false, false, EPI>(p, a, s);
    else if (!p.a_mn && p.b_mn) tg_launch_one<BN, false, true, EPI>(p, a, s);
    else tg_launch_one<BN, true, true, EPI>(p, a, s);
}

template <int EPI>
void tg_launch_epi(const TgPlan &p, const TgArgs &a, cudaStream_t s) {
    if (p.BN == 256) tg_launch_bn<256, EPI>(p, a, s);
    else if (p.BN == 128) tg_launch_bn<128, EPI>(p, a, s);
    else tg_launch_bn<64, EPI>(p, a, s);
}

}  // namespace

bool make_tg_plan(TgPlan &p, int epi, const void *A, bool a_mn, const void *B, bool b_mn, int M, int N, int R,
                  void *out, int ldo, const float *bias, const void *mask, std::string &why) {
    if (M <= 0 || N <= 0 || R <= 0) { why = "empty training GEMM"; return false; }
    if (N % 64 != 0) { why = "training GEMM: N not a multiple of 64"; return false; }
    if (a_mn && !b_mn) { why = "training GEMM: layout pair not built"; return false; }
    // the widest column tile that still gives three tiles for every four SMs; narrower tiles
    // before a split reduction (a split writes FP32 partial tiles and needs a reduction
    // kernel: FC1's forward of the training step went from 32 tiles x 4 splits to 128 tiles)
    {
        const int mt = (M + BM - 1) / BM, want = 3 * num_sms() / 4;
        p.BN = 64;
        for (int bn : {256, 128})
            if (N % bn == 0 && mt * (N / bn) >= want) { p.BN = bn; break; }
    }
    p.epi = epi;
    p.a_mn = a_mn;
    p.b_mn = b_mn;
    p.M = M;
    p.N = N;
    p.R = R;
    p.ldo = ldo;
    p.bias = bias;
    p.mask = mask;
    p.out = out;
    p.stages = p.BN == 256 ? 4 : p.BN == 128 ? 6 : 8;
    // A(m, r): K-major stored [M][R] (box 64 r x 128 m), MN-major stored [R][M] (box 64 m x 64 r)
    if (!a_mn) {
        if (!encode_map_2d(p.tA, SIMNET_BF16, A, (uint64_t)R, (uint64_t)M, 64, 128, why)) return false;
    } else {
        if (!encode_map_2d(p.tA, SIMNET_BF16, A, (uint64_t)M, (uint64_t)R, 64, 64, why)) return false;
    }
    if (!b_mn) {
        if (!encode_map_2d(p.tB, SIMNET_BF16, B, (uint64_t)R, (uint64_t)N, 64, (uint32_t)p.BN, why)) return false;
    } else {
        if (!encode_map_2d(p.tB, SIMNET_BF16, B, (uint64_t)N, (uint64_t)R, 64, 64, why)) return false;
    }
    p.m_tiles = (M + BM - 1) / BM;
    p.n_tiles_n = N / p.BN;
    const int KB = (R + 63) / 64, base = p.m_tiles * p.n_tiles_n, sms = num_sms();
    p.splits = 1;
    p.kb_per_split = KB;
    if ((epi == TG_WGRAD || epi == TG_FWD_F32) && base < 3 * sms / 4) {   // split the reduction until the tiles fill the GPU
        int splits = std::min(KB, (sms + base - 1) / base);
        p.kb_per_split = (KB + splits - 1) / splits;
        p.splits = (KB + p.kb_per_split - 1) / p.kb_per_split;
    }
    const int items = base * p.splits;
    p.grid = std::min(items, sms);
    p.smem = (size_t)p.stages * (A_BYTES + p.BN * ROW_BYTES) + 1024 + (2 * p.stages + 5) * 8 + 16;
    p.ready = true;
    return true;
}

void launch_tg(const TgPlan &p, int64_t spin_ns, int32_t *status, cudaStream_t s) {
    TgArgs a;
    a.bias = p.bias;
    a.mask = reinterpret_cast<const __nv_bfloat16 *>(p.mask);
    a.out = p.out;
    a.part = tg_part_floats(p) ? p.part : nullptr;
    a.M = p.M;
    a.N = p.N;
    a.R = p.R;
    a.ldo = p.ldo;
    a.n_tiles_n = p.n_tiles_n;
    a.m_tiles = p.m_tiles;
    a.splits = p.splits;
    a.kb_per_split = p.kb_per_split;
    a.spin_ns = spin_ns;
    a.status = status;
    switch (p.epi) {
        case TG_FWD_BF16: tg_launch_epi<TG_FWD_BF16>(p, a, s); break;
        case TG_FWD_F32: tg_launch_epi<TG_FWD_F32>(p, a, s); break;
        case TG_DGRAD: tg_launch_epi<TG_DGRAD>(p, a, s); break;
        default: tg_launch_epi<TG_WGRAD>(p, a, s); break;
    }
    if (a.part) {
        const bool fwd = p.epi == TG_FWD_F32;
        const int64_t count = fwd ? (int64_t)p.M * p.N : (int64_t)p.N * p.ldo;
        if (count % 4 == 0)
            tg_reduce4_kernel<<<(unsigned)((count / 4 + 31) / 32), 256, 0, s>>>(
                a.part, p.splits, count, reinterpret_cast<float *>(p.out), fwd ? p.bias : nullptr, p.N, fwd ? 1 : 0);
        else
            tg_reduce_kernel<<<(unsigned)((count + 31) / 32), 256, 0, s>>>(a.part, p.splits, count,
                                                                           reinterpret_cast<float *>(p.out),
                                                                           fwd ? p.bias : nullptr, p.N, fwd ? 1 : 0);
    }
}

}  // namespace simnet
