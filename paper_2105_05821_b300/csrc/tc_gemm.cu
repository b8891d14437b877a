// tc_gemm.cu -- the CNN layers (Sec. 2.3) as tcgen05 tensor-core GEMMs on sm_103a.
//
// C[M,N] = act(A[M,K] * B[N,K]^T * scale[n] + bias[n]) * oscale[n], A and B
// K-major.  A k=2/stride-2 convolution is exactly this GEMM on the contiguous
// reshape [rows/2, 2*C_in] of its input, and FC1 is it on the flatten.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0     TMA producer: A and B tiles (128-byte swizzle) into an S-stage
//              shared-memory ring, completion on `full` mbarriers;
//   warp 1     MMA issuer: one thread issues tcgen05.mma (kind::f16 for BF16,
//              kind::f8f6f4 for FP8 e4m3) into a TMEM accumulator; commits free
//              ring stages (`empty`) and hand finished accumulators to the
//              epilogue (`tfull`);
//   warps 2-5  epilogue: tcgen05.ld 32 columns at a time, scale, bias, ReLU,
//              requantise, store; then release the accumulator (`tempty`).
// Two TMEM accumulators let the epilogue of one tile overlap the MMAs of the
// next.  Every wait is bounded by a globaltimer limit: on expiry the kernel
// records a timeout in the device status word, stops issuing work, waits
// (bounded) for its own TMA copies still in flight, frees TMEM and returns.
#include <cstdio>
#include <cudaTypedefs.h>
#include <mutex>

#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace simnet {

namespace {

using namespace tcx;

enum OutKind { OUT_BF16 = 0, OUT_F32 = 1, OUT_FP8 = 2, OUT_FC2PART = 3, OUT_FC2HYB = 4, OUT_FC2P3 = 5, OUT_FC2P33 = 6 };
// FC2 outputs folded by the generic (L1-read) epilogue of an output kind, 0 if none
template <int OUT> constexpr int fc2_outs() {
    return OUT == OUT_FC2HYB ? 22 : OUT == OUT_FC2P3 ? 3 : OUT == OUT_FC2P33 ? 33 : 0;
}

struct TcArgs {
    const float *bias, *scale, *oscale, *w2;
    const void *resid;         // [M][N] in the output precision, added before the activation, or null
    void *out;                 // [M][N] activations, or FC2 partials [2 * n_tiles_n][part_stride][2 or 22] float
    const int32_t *count;
    int m_mult, m_cap, N, K, relu, n_tiles_n, part_stride, prm_floats;
    int64_t spin_ns;
    int32_t *status;
};

// Per-launch shared-memory layout (after the 1024-aligned stage ring):
// barriers | TMEM slot + abort flag | per-column parameters | epilogue staging.
template <int BN, int STAGES, int OUT>
struct TcLayout {
    static constexpr int B_BYTES = BN * ROW_BYTES;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int RING = STAGES * STAGE_BYTES;
    static constexpr int BARS = (2 * STAGES + 4) * 8 + 16;
    static constexpr int OUT_ES = OUT == OUT_F32 ? 4 : OUT == OUT_BF16 ? 2 : 1;
    static constexpr int CHUNK_BYTES = 32 * OUT_ES;        // 32 output columns of one row
    static constexpr int STAGE_ROW = CHUNK_BYTES + 16;     // padded: conflict-free 16-byte stores
    static constexpr int EPI_WARPS = 8;                    // two per TMEM lane quadrant
    static constexpr int STAGING = OUT >= OUT_FC2PART ? 0 : EPI_WARPS * 32 * STAGE_ROW;
};

template <int BN, int STAGES, bool FP8, int OUT>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const TcArgs args) {
    using L = TcLayout<BN, STAGES, OUT>;
    constexpr int BK = FP8 ? 128 : 64;         // elements per 128-byte row
    constexpr int KSTEP_DESC = 32 >> 4;       // one MMA consumes 32 bytes of K
    constexpr uint32_t TMEM_COLS = 2 * BN;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::RING);
    // bars[0..S) full, [S..2S) empty, [2S..2S+2) tfull, [2S+2..2S+4) tempty
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *prm = reinterpret_cast<float *>(smem + L::RING + L::BARS);   // bias | scale | oscale | w2 (each N, w2 2N)
    // (the hybrid head's 22 FC2 rows are read through L1 instead of being staged)
    const int N = args.N;
    float *s_bias = prm, *s_scale = prm + N, *s_oscale = prm + 2 * N, *s_w2 = prm + 3 * N;
    uint8_t *staging = smem + L::RING + L::BARS + args.prm_floats * 4;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t smem_base = smem_u32(smem);
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto tfull = [&](int a) { return smem_u32(&bars[2 * STAGES + a]); };
    auto tempty = [&](int a) { return smem_u32(&bars[2 * STAGES + 2 + a]); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), 32 * L::EPI_WARPS);
        }
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
    // per-column parameters are weights: they do not depend on the previous kernel
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        s_bias[i] = args.bias[i];
        if (args.scale) s_scale[i] = args.scale[i];
        if (args.oscale) s_oscale[i] = args.oscale[i];
        if constexpr (OUT == OUT_FC2PART) {
            s_w2[i] = args.w2[i];
            s_w2[N + i] = args.w2[N + i];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // everything below reads what earlier kernels in the stream wrote
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const int M = min(*args.count * args.m_mult, args.m_cap);
    const int m_tiles = (M + BM - 1) / BM;
    const int n_tiles = m_tiles * args.n_tiles_n;
    const int KB = args.K / BK;
    const int64_t lim = args.spin_ns;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const int m0 = (t / args.n_tiles_n) * BM, n0 = (t % args.n_tiles_n) * BN;
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(empty(s), ph ^ 1u, lim, abort_flag, args.status)) { ok = false; break; }
                    const uint32_t sa = smem_base + s * L::STAGE_BYTES;
                    mbar_expect_tx(full(s), L::STAGE_BYTES);
                    tma_load_2d(sa, &tA, full(s), kb * BK, m0);
                    tma_load_2d(sa + A_BYTES, &tB, full(s), kb * BK, n0);
                }
            }
            if (!ok) {  // let the copies already issued land before the CTA's memory is released
                for (int j = max(0, it - STAGES); j < it; j++) {
                    volatile int never = 0;
                    mbar_wait(full(j % STAGES), (uint32_t)(j / STAGES) & 1u, lim, &never, args.status);
                }
            }
        }
    } else if (warp == 1) {
        {   // the whole warp runs the issue loop, one elected lane issues (umma_warp)
            int it = 0, tc = 0;
            bool ok = true;
            constexpr uint32_t ID = idesc<BN, FP8>();
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, tc++) {
                const int acc = tc & 1;
                const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait(tempty(acc), aph ^ 1u, lim, abort_flag, args.status))) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!__all_sync(0xffffffffu, mbar_wait(full(s), ph, lim, abort_flag, args.status))) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_base + s * L::STAGE_BYTES;
                    const uint64_t ad = sdesc(sa), bd = sdesc(sa + A_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        umma_warp<FP8>(d, ad + (uint64_t)(k * KSTEP_DESC), bd + (uint64_t)(k * KSTEP_DESC), ID,
                                       (kb | k) != 0 ? 1u : 0u);
                    umma_commit_warp(empty(s));
                }
                if (ok) umma_commit_warp(tfull(acc));
            }
        }
        __syncwarp();
    } else {
        // epilogue: warps 2..9.  Warp w reads TMEM lanes 32*(w%4) .. +31 (= tile rows)
        // and the column half (w-2)/4 of the tile.
        const int q = warp & 3, half = (warp - 2) >> 2;
        constexpr int CPW = BN / 64;               // 32-column chunks per warp
        uint8_t *stg = staging + (warp - 2) * 32 * L::STAGE_ROW;
        const size_t ldc_bytes = (size_t)N * L::OUT_ES;
        int tc = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, tc++) {
            const int mt = t / args.n_tiles_n, nt = t % args.n_tiles_n;
            const int m0 = mt * BM, n0 = nt * BN;
            const int acc = tc & 1;
            const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
            if (!mbar_wait(tfull(acc), aph, lim, abort_flag, args.status)) break;
            tc_fence_after();
            const int row = m0 + q * 32 + lane;
            const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + half * (BN / 2));
            float pf = 0.f, pe = 0.f;
            constexpr int NH = fc2_outs<OUT>() > 0 ? fc2_outs<OUT>() : 1;
            float ph[NH];
#pragma unroll
            for (int o = 0; o < NH; o++) ph[o] = 0.f;
#pragma unroll 1
            for (int c = 0; c < CPW; c++) {
                uint32_t r[32];
                tmem_ld32(tbase + (uint32_t)(c * 32), r);
                const int col0 = n0 + half * (BN / 2) + c * 32;
                float v[32];
                // residual block: the shortcut rows (same layout as the output)
                float rs[32];
#pragma unroll
                for (int j = 0; j < 32; j++) rs[j] = 0.f;
                if constexpr (OUT == OUT_BF16) {
                    if (args.resid && row < M) {
                        const uint4 *rp = reinterpret_cast<const uint4 *>(
                            reinterpret_cast<const __nv_bfloat16 *>(args.resid) + (size_t)row * N + col0);
#pragma unroll
                        for (int q4 = 0; q4 < 4; q4++) {
                            const uint4 u = rp[q4];
                            const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w4[h]));
                                rs[8 * q4 + 2 * h] = f.x;
                                rs[8 * q4 + 2 * h + 1] = f.y;
                            }
                        }
                    }
                } else if constexpr (OUT == OUT_F32) {
                    if (args.resid && row < M) {
                        const float4 *rp =
                            reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(args.resid) + (size_t)row * N + col0);
#pragma unroll
                        for (int q4 = 0; q4 < 8; q4++) {
                            const float4 f = rp[q4];
                            rs[4 * q4] = f.x;
                            rs[4 * q4 + 1] = f.y;
                            rs[4 * q4 + 2] = f.z;
                            rs[4 * q4 + 3] = f.w;
                        }
                    }
                }
#pragma unroll
                for (int j4 = 0; j4 < 8; j4++) {
                    const float4 bb = *reinterpret_cast<const float4 *>(s_bias + col0 + 4 * j4);
                    float4 sc = make_float4(1.f, 1.f, 1.f, 1.f), os = sc;
                    if constexpr (FP8) {
                        sc = *reinterpret_cast<const float4 *>(s_scale + col0 + 4 * j4);
                        if (args.oscale) os = *reinterpret_cast<const float4 *>(s_oscale + col0 + 4 * j4);
                    }
                    const float b4[4] = {bb.x, bb.y, bb.z, bb.w}, s4[4] = {sc.x, sc.y, sc.z, sc.w},
                                o4[4] = {os.x, os.y, os.z, os.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        float x = __uint_as_float(r[4 * j4 + e]);
                        if constexpr (FP8) x *= s4[e];
                        x += b4[e] + rs[4 * j4 + e];
                        if (args.relu) x = fmaxf(x, 0.f);
                        if constexpr (FP8) x *= o4[e];
                        v[4 * j4 + e] = x;
                    }
                }
                if constexpr (OUT == OUT_FC2PART) {
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 wf = *reinterpret_cast<const float4 *>(s_w2 + col0 + 4 * j4);
                        const float4 we = *reinterpret_cast<const float4 *>(s_w2 + N + col0 + 4 * j4);
                        pf = fmaf(v[4 * j4], wf.x, pf); pf = fmaf(v[4 * j4 + 1], wf.y, pf);
                        pf = fmaf(v[4 * j4 + 2], wf.z, pf); pf = fmaf(v[4 * j4 + 3], wf.w, pf);
                        pe = fmaf(v[4 * j4], we.x, pe); pe = fmaf(v[4 * j4 + 1], we.y, pe);
                        pe = fmaf(v[4 * j4 + 2], we.z, pe); pe = fmaf(v[4 * j4 + 3], we.w, pe);
                    }
                } else if constexpr (fc2_outs<OUT>() > 0) {
                    // every lane reads the same FC2 row segment: L1 broadcasts
#pragma unroll
                    for (int o = 0; o < NH; o++) {
                        const float4 *wr = reinterpret_cast<const float4 *>(args.w2 + (size_t)o * N + col0);
#pragma unroll
                        for (int j4 = 0; j4 < 8; j4++) {
                            const float4 w = __ldg(wr + j4);
                            ph[o] = fmaf(v[4 * j4], w.x, ph[o]); ph[o] = fmaf(v[4 * j4 + 1], w.y, ph[o]);
                            ph[o] = fmaf(v[4 * j4 + 2], w.z, ph[o]); ph[o] = fmaf(v[4 * j4 + 3], w.w, ph[o]);
                        }
                    }
                } else {
                    // this thread's row segment -> padded staging row `lane`
                    uint4 *dst = reinterpret_cast<uint4 *>(stg + lane * L::STAGE_ROW);
                    if constexpr (OUT == OUT_F32) {
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            dst[j] = make_uint4(__float_as_uint(v[4 * j]), __float_as_uint(v[4 * j + 1]),
                                                __float_as_uint(v[4 * j + 2]), __float_as_uint(v[4 * j + 3]));
                    } else if constexpr (OUT == OUT_BF16) {
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
                    } else {
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
                    }
                    __syncwarp();
                    // coalesced copy-out: U lanes per row, 32/U rows per pass
                    constexpr int U = L::CHUNK_BYTES / 16, RPP = 32 / U;
                    const int rr = lane / U, u = lane % U;
                    uint8_t *gbase = reinterpret_cast<uint8_t *>(args.out) + (size_t)col0 * L::OUT_ES + u * 16;
#pragma unroll
                    for (int pass = 0; pass < U; pass++) {
                        const int r_in = pass * RPP + rr;
                        const int grow = m0 + q * 32 + r_in;
                        const uint4 val = *reinterpret_cast<const uint4 *>(stg + r_in * L::STAGE_ROW + u * 16);
                        if (grow < M) *reinterpret_cast<uint4 *>(gbase + (size_t)grow * ldc_bytes) = val;
                    }
                    __syncwarp();
                }
            }
            if constexpr (OUT == OUT_FC2PART) {  // one partial per (column block, half)
                if (row < M)
                    reinterpret_cast<float2 *>(args.out)[(size_t)(2 * nt + half) * args.part_stride + row] =
                        make_float2(pf, pe);
            }
            if constexpr (fc2_outs<OUT>() > 0) {
                if (row < M) {
                    float *dst = reinterpret_cast<float *>(args.out) +
                                 ((size_t)(2 * nt + half) * args.part_stride + row) * NH;
#pragma unroll
                    for (int o = 0; o < NH; o++) dst[o] = ph[o];
                }
            }
            tc_fence_before();
            mbar_arrive(tempty(acc));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_2d(CUtensorMap &m, int prec, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
               uint32_t box_outer, std::string &why) {
    auto fn = encode_fn();
    if (!fn) { why = "cuTensorMapEncodeTiled unavailable"; return false; }
    const uint64_t es = prec == SIMNET_BF16 ? 2 : 1;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * es};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&m, prec == SIMNET_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[96];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled error %d", (int)r);
        why = buf;
        return false;
    }
    return true;
}

template <int BN, int STAGES, bool FP8, int OUT>
void launch_one(const TcPlan &p, const TcArgs &a, cudaStream_t s) {
    static size_t attr = 0;
    auto k = tc_gemm_kernel<BN, STAGES, FP8, OUT>;
    if (attr < p.smem) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        attr = p.smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.grid);
    cfg.blockDim = dim3(320);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = p.pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, p.tA, p.tB, a);
}

template <bool FP8, int OUT>
void dispatch(const TcPlan &p, const TcArgs &a, cudaStream_t s) {
    switch (p.BN) {
        case 64: launch_one<64, 6, FP8, OUT>(p, a, s); break;
        case 128: launch_one<128, 5, FP8, OUT>(p, a, s); break;
        default: launch_one<256, 3, FP8, OUT>(p, a, s); break;
    }
}

int stages_for(int BN) { return BN == 64 ? 6 : BN == 128 ? 5 : 3; }

int out_es(int out_kind, int prec) {
    return out_kind == TC_OUT_F32 ? 4 : out_kind >= TC_OUT_PART ? 0 : (prec == SIMNET_BF16 ? 2 : 1);
}

}  // namespace

bool encode_map_2d(CUtensorMap &m, int prec, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                   uint32_t box_outer, std::string &why) {
    return encode_2d(m, prec, base, inner, outer, box_inner, box_outer, why);
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

static void finish_plan(TcPlan &p) {
    p.stages = stages_for(p.BN);
    const int es = out_es(p.out_kind, p.prec);
    const size_t staging = p.out_kind >= TC_OUT_PART ? 0 : (size_t)8 * 32 * (32 * es + 16);
    p.smem = (size_t)p.stages * (A_BYTES + p.BN * ROW_BYTES) + 1024 + ((2 * p.stages + 4) * 8 + 16) +
             (size_t)p.prm_floats * 4 + staging;
    const int m_tiles = (p.m_cap + BM - 1) / BM;
    const int tiles = m_tiles * (p.N / p.BN);
    p.grid = tiles < num_sms() ? (tiles > 0 ? tiles : 1) : num_sms();
}

bool make_tc_plan(TcPlan &p, int prec, const void *in, const GemmLayer &g, void *out, int out_kind, int m_cap,
                  int64_t spin_ns, int32_t *status, bool pdl, std::string &why, const void *resid) {
    if (p.ready && p.prec == prec && p.in == in && p.out == out && p.m_cap == m_cap && p.K == g.K && p.N == g.N &&
        p.out_kind == out_kind && p.status == status && p.pdl == pdl && p.wB == g.B && p.resid == resid)
        return true;
    if (resid && !(out_kind == TC_OUT_ACT && prec == SIMNET_BF16) && out_kind != TC_OUT_F32) {
        why = "a shortcut is added only to BF16 or FP32 outputs";
        return false;
    }
    p.resid = resid;
    const int BK = prec == SIMNET_BF16 ? 64 : 128;
    if (g.K % BK != 0 || g.N % 64 != 0) { why = "K or N not a multiple of the tile"; return false; }
    p.prec = prec;
    p.in = in;
    p.out = out;
    p.wB = g.B;
    p.m_cap = m_cap;
    p.K = g.K;
    p.N = g.N;
    p.out_kind = out_kind;
    p.spin_ns = spin_ns;
    p.status = status;
    p.pdl = pdl;
    p.prm_floats = g.N * 3 + (out_kind == TC_OUT_PART ? 2 * g.N : 0);
    // widest tile that still gives every SM two tiles; else the narrowest
    const int m_tiles = (m_cap + BM - 1) / BM;
    p.BN = 64;
    for (int bn : {256, 128}) {
        if (g.N % bn == 0 && (int64_t)m_tiles * (g.N / bn) >= 2 * num_sms()) { p.BN = bn; break; }
    }
    finish_plan(p);
    if (p.smem > 232448) { why = "shared memory budget exceeded"; return false; }
    if (!encode_2d(p.tA, prec, in, (uint64_t)g.K, (uint64_t)m_cap, BK, BM, why)) return false;
    if (!encode_2d(p.tB, prec, g.B, (uint64_t)g.K, (uint64_t)g.N, BK, p.BN, why)) return false;
    p.ready = true;
    return true;
}

bool retune_tc_plan(TcPlan &p, const GemmLayer &g, int BN, std::string &why) {
    if (!p.ready || g.N % BN != 0 || !(BN == 64 || BN == 128 || BN == 256)) { why = "bad tile"; return false; }
    p.BN = BN;
    finish_plan(p);
    if (p.smem > 232448) { why = "shared memory budget exceeded"; return false; }
    const int BK = p.prec == SIMNET_BF16 ? 64 : 128;
    return encode_2d(p.tB, p.prec, g.B, (uint64_t)g.K, (uint64_t)g.N, BK, p.BN, why);
}

void launch_tc_gemm(const TcPlan &p, const GemmLayer &g, const int32_t *count, const float *w2, cudaStream_t s) {
    TcArgs a;
    a.resid = p.resid;
    a.bias = g.bias;
    a.scale = g.scale;
    a.oscale = g.oscale;
    a.w2 = w2;
    a.out = p.out;
    a.count = count;
    a.m_mult = g.m_mult;
    a.m_cap = p.m_cap;
    a.N = g.N;
    a.K = g.K;
    a.relu = g.relu;
    a.n_tiles_n = g.N / p.BN;
    a.part_stride = p.m_cap;
    a.prm_floats = p.prm_floats;
    a.spin_ns = p.spin_ns;
    a.status = p.status;
    const bool fp8 = p.prec != SIMNET_BF16;
    switch (p.out_kind) {
        case TC_OUT_F32:
            if (fp8) dispatch<true, OUT_F32>(p, a, s);
            else dispatch<false, OUT_F32>(p, a, s);
            break;
        case TC_OUT_PART:
            if (fp8) dispatch<true, OUT_FC2PART>(p, a, s);
            else dispatch<false, OUT_FC2PART>(p, a, s);
            break;
        case TC_OUT_PART_HYBRID:
            if (fp8) dispatch<true, OUT_FC2HYB>(p, a, s);
            else dispatch<false, OUT_FC2HYB>(p, a, s);
            break;
        case TC_OUT_PART3:
            if (fp8) dispatch<true, OUT_FC2P3>(p, a, s);
            else dispatch<false, OUT_FC2P3>(p, a, s);
            break;
        case TC_OUT_PART33:
            if (fp8) dispatch<true, OUT_FC2P33>(p, a, s);
            else dispatch<false, OUT_FC2P33>(p, a, s);
            break;
        default:
            if (fp8) dispatch<true, OUT_FP8>(p, a, s);
            else dispatch<false, OUT_BF16>(p, a, s);
    }
}

}  // namespace simnet
