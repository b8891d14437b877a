// tc_ptx.cuh -- inline PTX wrappers for tcgen05 MMAs, TMEM, TMA and mbarriers
// (sm_103a), shared by the tensor-core kernels.  Every wait is bounded.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace simnet {
namespace tcx {

constexpr int BM = 128;
constexpr int ROW_BYTES = 128;  // one K-block row = one 128-byte swizzle row
constexpr int A_BYTES = BM * ROW_BYTES;

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

// Non-blocking test of a phase (inline: the common case of a phase that has
// already completed costs no call).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false if it gave up (or another role did).
__device__ __noinline__ inline bool mbar_wait_slow(uint32_t bar, uint32_t parity, int64_t limit,
                                                   volatile int *abort_flag, int32_t *status) {
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int64_t limit, volatile int *abort_flag,
                                          int32_t *status) {
    if (mbar_test(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, limit, abort_flag, status);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Prefetch of a tile of a tensor into L2 (no shared memory, no barrier).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
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

// The same MMA from a converged warp: every lane runs the issue loop (so the
// operands are warp-uniform values) and one elected lane issues.  A lone
// thread in a divergent branch issued an MMA every ~95 cycles on this GPU,
// a whole warp every ~64.
template <bool FP8>
__device__ __forceinline__ void umma_warp(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accum) {
    if constexpr (FP8) {
        asm volatile(
            "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(id), "r"(accum));
    } else {
        asm volatile(
            "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(id), "r"(accum));
    }
}
// Low word of sdesc(saddr); the high word (stride 1024, version, 128-byte swizzle) is
// kSdescHi for every operand of these kernels.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t saddr) { return ((saddr & 0x3FFFFu) >> 4) | (1u << 16); }
constexpr uint32_t kSdescHi = (1024u >> 4) | (1u << 14) | (2u << 29);
// umma_warp on descriptors given by their low words (32-bit arithmetic on the issue path).
template <bool FP8>
__device__ __forceinline__ void umma_lo(uint32_t tmem_d, uint32_t a_lo, uint32_t b_lo, uint32_t id, uint32_t accum) {
    if constexpr (FP8) {
        asm volatile(
            "{\n .reg .pred e, p;\n .reg .b64 da, db;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %5};\n"
            " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
            "r"(a_lo), "r"(b_lo), "r"(id), "r"(accum), "n"(kSdescHi));
    } else {
        asm volatile(
            "{\n .reg .pred e, p;\n .reg .b64 da, db;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %5};\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
            "r"(a_lo), "r"(b_lo), "r"(id), "r"(accum), "n"(kSdescHi));
    }
}
// High word of a descriptor of a K-major operand with 64-byte rows, 64-byte swizzle
// (8-row groups 512 bytes apart); its low word is sdesc_lo of the start address.
constexpr uint32_t kSdescHi64 = (512u >> 4) | (1u << 14) | (4u << 29);
// umma_lo with A's high word given (A with 64-byte swizzle, B with 128-byte swizzle).
template <bool FP8>
__device__ __forceinline__ void umma_lo_a(uint32_t tmem_d, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t id,
                                          uint32_t accum) {
    if constexpr (FP8) {
        asm volatile(
            "{\n .reg .pred e, p;\n .reg .b64 da, db;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %6};\n"
            " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
            "r"(a_lo), "r"(b_lo), "r"(id), "r"(accum), "r"(a_hi), "n"(kSdescHi));
    } else {
        asm volatile(
            "{\n .reg .pred e, p;\n .reg .b64 da, db;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %6};\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
            "r"(a_lo), "r"(b_lo), "r"(id), "r"(accum), "r"(a_hi), "n"(kSdescHi));
    }
}
// MMA with A in tensor memory (rows on lanes 0..127, K packed along the columns: two
// BF16 or four E4M3 values to a 32-bit column, lowest K in the low bits) and B a
// K-major 128-byte-swizzled shared-memory operand given by its descriptor's low word.
template <bool FP8>
__device__ __forceinline__ void umma_ts(uint32_t tmem_d, uint32_t tmem_a, uint32_t b_lo, uint32_t id, uint32_t accum) {
    if constexpr (FP8) {
        asm volatile(
            "{\n .reg .pred e, p;\n .reg .b64 db;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " mov.b64 db, {%2, %5};\n"
            " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], db, %3, p;\n}\n" ::"r"(tmem_d),
            "r"(tmem_a), "r"(b_lo), "r"(id), "r"(accum), "n"(kSdescHi));
    } else {
        asm volatile(
            "{\n .reg .pred e, p;\n .reg .b64 db;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " mov.b64 db, {%2, %5};\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], db, %3, p;\n}\n" ::"r"(tmem_d),
            "r"(tmem_a), "r"(b_lo), "r"(id), "r"(accum), "n"(kSdescHi));
    }
}
// Commit from a converged warp (one elected lane).
__device__ __forceinline__ void umma_commit_warp(uint32_t bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
        : "memory");
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

// 32 lanes x 16 columns of 32-bit words into tensor memory (thread i: lane base + i),
// complete when it returns.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 lanes x 64 columns in one load, complete when it returns.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
}
// 32 lanes x 32 columns into tensor memory; tmem_st_wait() completes it.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}
// max(x, 0) for two values rounded to BF16 (lo in the low half): the conversion
// applies the ReLU, which commutes with round-to-nearest.
__device__ __forceinline__ uint32_t bf16x2_relu(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// The same for E4M3 with saturation to the finite range (16 bits, lo in the low byte).
__device__ __forceinline__ uint32_t e4m3x2_relu(float lo, float hi) {
    unsigned short d;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
    return (uint32_t)d;
}

// Instruction descriptor with N chosen at run time.
__device__ __forceinline__ uint32_t idesc_rt(int BN, bool fp8) {
    return (1u << 4) | ((fp8 ? 0u : 1u) << 7) | ((fp8 ? 0u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

}  // namespace tcx
}  // namespace simnet
