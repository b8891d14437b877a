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

namespace simnet {

namespace {

constexpr int BM = 128;
constexpr int ROW_BYTES = 128;  // one K-block row = one 128-byte swizzle row
constexpr int A_BYTES = BM * ROW_BYTES;

enum OutKind { OUT_BF16 = 0, OUT_F32 = 1, OUT_FP8 = 2 };

struct TcArgs {
    const float *bias, *scale, *oscale;
    void *out;
    const int32_t *count;
    int m_mult, m_cap, N, K, relu, n_tiles_n;
    int64_t spin_ns;
    int32_t *status;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false if it gave up (or another role did).
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int64_t limit, volatile int *abort_flag,
                                       int32_t *status) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(gtimer() - t0) > limit) {
            *abort_flag = 1;
            atomicExch(status, kStatusTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte
// swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = BN;
// BF16 x BF16 (kind::f16) or E4M3 x E4M3 (kind::f8f6f4).
template <int BN, bool FP8>
__device__ __forceinline__ constexpr uint32_t idesc() {
    return (1u << 4) | ((FP8 ? 0u : 1u) << 7) | ((FP8 ? 0u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

template <bool FP8>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accum) {
    if constexpr (FP8) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem_d),
            "l"(a), "l"(b), "r"(id), "r"(accum));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem_d),
            "l"(a), "l"(b), "r"(id), "r"(accum));
    }
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN, int STAGES, bool FP8, int OUT>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const TcArgs args) {
    constexpr int B_BYTES = BN * ROW_BYTES;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr int BK = FP8 ? 128 : 64;         // elements per 128-byte row
    constexpr int KSTEP_DESC = 32 >> 4;       // one MMA consumes 32 bytes of K
    constexpr uint32_t TMEM_COLS = 2 * BN;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    // bars[0..S) full, [S..2S) empty, [2S..2S+2) tfull, [2S+2..2S+4) tempty
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

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
            mbar_init(tempty(a), 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
                    const uint32_t sa = smem_base + s * STAGE_BYTES;
                    mbar_expect_tx(full(s), STAGE_BYTES);
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
        if (lane == 0) {
            int it = 0, tc = 0;
            bool ok = true;
            constexpr uint32_t ID = idesc<BN, FP8>();
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, tc++) {
                const int acc = tc & 1;
                const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
                if (!mbar_wait(tempty(acc), aph ^ 1u, lim, abort_flag, args.status)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(full(s), ph, lim, abort_flag, args.status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_base + s * STAGE_BYTES;
                    const uint64_t ad = sdesc(sa), bd = sdesc(sa + A_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        umma<FP8>(d, ad + (uint64_t)(k * KSTEP_DESC), bd + (uint64_t)(k * KSTEP_DESC), ID,
                                  (kb | k) != 0 ? 1u : 0u);
                    umma_commit(empty(s));
                }
                if (ok) umma_commit(tfull(acc));
            }
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 = tile rows of the same range
        const int q = warp & 3;
        const int ldc = args.N;
        int tc = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, tc++) {
            const int m0 = (t / args.n_tiles_n) * BM, n0 = (t % args.n_tiles_n) * BN;
            const int acc = tc & 1;
            const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
            if (!mbar_wait(tfull(acc), aph, lim, abort_flag, args.status)) break;
            tc_fence_after();
            const int row = m0 + q * 32 + lane;
            const bool row_ok = row < M;
#pragma unroll 1
            for (int c = 0; c < BN / 32; c++) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c * 32), r);
                const int col0 = n0 + c * 32;
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    float x = __uint_as_float(r[j]);
                    if (args.scale) x *= __ldg(args.scale + col0 + j);
                    x += __ldg(args.bias + col0 + j);
                    if (args.relu) x = fmaxf(x, 0.f);
                    if (args.oscale) x *= __ldg(args.oscale + col0 + j);
                    v[j] = x;
                }
                if (row_ok) {
                    if constexpr (OUT == OUT_F32) {
                        float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(args.out) + (size_t)row * ldc + col0);
#pragma unroll
                        for (int j = 0; j < 8; j++) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    } else if constexpr (OUT == OUT_BF16) {
                        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(args.out) + (size_t)row * ldc + col0);
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
                        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(args.out) + (size_t)row * ldc + col0);
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
    static bool attr = false;
    auto k = tc_gemm_kernel<BN, STAGES, FP8, OUT>;
    if (!attr) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        attr = true;
    }
    k<<<p.grid, 192, p.smem, s>>>(p.tA, p.tB, a);
}

template <bool FP8, int OUT>
void dispatch(const TcPlan &p, const TcArgs &a, cudaStream_t s) {
    switch (p.BN) {
        case 64: launch_one<64, 8, FP8, OUT>(p, a, s); break;
        case 128: launch_one<128, 6, FP8, OUT>(p, a, s); break;
        default: launch_one<256, 4, FP8, OUT>(p, a, s); break;
    }
}

int stages_for(int BN) { return BN == 64 ? 8 : BN == 128 ? 6 : 4; }

}  // namespace

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
    p.smem = (size_t)p.stages * (A_BYTES + p.BN * ROW_BYTES) + 1024 + 256;
    const int m_tiles = (p.m_cap + BM - 1) / BM;
    const int tiles = m_tiles * (p.N / p.BN);
    p.grid = tiles < num_sms() ? (tiles > 0 ? tiles : 1) : num_sms();
}

bool make_tc_plan(TcPlan &p, int prec, const void *in, const GemmLayer &g, void *out, bool out_f32, int m_cap,
                  int64_t spin_ns, int32_t *status, std::string &why) {
    if (p.ready && p.prec == prec && p.in == in && p.out == out && p.m_cap == m_cap && p.K == g.K && p.N == g.N &&
        p.out_f32 == out_f32 && p.status == status)
        return true;
    const int BK = prec == SIMNET_BF16 ? 64 : 128;
    if (g.K % BK != 0 || g.N % 64 != 0) { why = "K or N not a multiple of the tile"; return false; }
    p.prec = prec;
    p.in = in;
    p.out = out;
    p.m_cap = m_cap;
    p.K = g.K;
    p.N = g.N;
    p.out_f32 = out_f32;
    p.spin_ns = spin_ns;
    p.status = status;
    // widest tile that still gives every SM two tiles; else the narrowest
    const int m_tiles = (m_cap + BM - 1) / BM;
    p.BN = 64;
    for (int bn : {256, 128}) {
        if (g.N % bn == 0 && (int64_t)m_tiles * (g.N / bn) >= 2 * num_sms()) { p.BN = bn; break; }
    }
    finish_plan(p);
    if (!encode_2d(p.tA, prec, in, (uint64_t)g.K, (uint64_t)m_cap, BK, BM, why)) return false;
    if (!encode_2d(p.tB, prec, g.B, (uint64_t)g.K, (uint64_t)g.N, BK, p.BN, why)) return false;
    p.ready = true;
    return true;
}

bool retune_tc_plan(TcPlan &p, const GemmLayer &g, int BN, int stages, std::string &why) {
    (void)stages;
    if (!p.ready || g.N % BN != 0 || !(BN == 64 || BN == 128 || BN == 256)) { why = "bad tile"; return false; }
    p.BN = BN;
    finish_plan(p);
    const int BK = p.prec == SIMNET_BF16 ? 64 : 128;
    return encode_2d(p.tB, p.prec, g.B, (uint64_t)g.K, (uint64_t)g.N, BK, p.BN, why);
}

void launch_tc_gemm(const TcPlan &p, const void *in, const GemmLayer &g, void *out, bool out_f32,
                    const int32_t *count, int m_cap, cudaStream_t s) {
    (void)in;
    TcArgs a;
    a.bias = g.bias;
    a.scale = g.scale;
    a.oscale = g.oscale;
    a.out = out;
    a.count = count;
    a.m_mult = g.m_mult;
    a.m_cap = m_cap;
    a.N = g.N;
    a.K = g.K;
    a.relu = g.relu;
    a.n_tiles_n = g.N / p.BN;
    a.spin_ns = p.spin_ns;
    a.status = p.status;
    if (p.prec == SIMNET_BF16) {
        if (out_f32) dispatch<false, OUT_F32>(p, a, s);
        else dispatch<false, OUT_BF16>(p, a, s);
    } else {
        if (out_f32) dispatch<true, OUT_F32>(p, a, s);
        else dispatch<true, OUT_FP8>(p, a, s);
    }
}

}  // namespace simnet
