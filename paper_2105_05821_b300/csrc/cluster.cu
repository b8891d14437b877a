// cluster.cu -- the whole lock-step simulation of one simnet_simulate call as
// independent thread-block clusters (BF16 or FP8 e4m3 CNNs with 2 or 3 conv
// layers of 64 or 128 channels).
//
// Sub-traces never interact (Sec. 3.3), so a cluster of CS = 4 or 8 CTAs takes
// 128 batch slots for the whole call, 128 / CS per CTA, and needs no grid-wide
// synchronisation at all:
//   * each CTA keeps its slots' state in shared memory: position, curTick, the
//     processor-queue ring and its counters (Sec. 3.2), and the instruction
//     records, fetched two steps ahead with cp.async;
//   * per step the last-conv output positions below the cluster's padding
//     extent are processed in passes of up to 256 first-layer rows: a CTA
//     writes the feature rows (Sec. 2.2) of its slots that those positions
//     depend on straight into shared memory and runs the k=2 / stride-2 conv
//     pyramid on them (Sec. 2.3), one tcgen05 MMA per 128-row tile and layer
//     (rows as A, the layer's weights streamed by TMA as B, each CTA loading
//     its own copy, several panels to a pipeline stage); layer l's epilogue
//     writes layer l+1's operand in place, rows 2j and 2j+1 of a slot side by
//     side along K;
//   * the last conv layer's rows of all 128 slots are exchanged through
//     distributed shared memory by bulk copies, and every CTA accumulates FC1
//     for its 1 / CS of the hidden neurons in TMEM over the passes; positions
//     at or past the extent are constant rows whose FC1 contribution S[e] was
//     tabulated when the weights were loaded;
//   * the FC1 epilogue folds FC2 into per-slot partial sums that go to each
//     slot's owner CTA (st.async), where one thread per slot runs the head,
//     the clock and queue update and the drain (Eq. 1); the CTA then shares its
//     new extent with the cluster (st.async).
// Every wait is bounded (globaltimer); an expired wait records a timeout and
// the CTA leaves at the next step boundary.  Leaving is deterministic: each CTA
// counts what it sent every peer (extents, partial sums, row copies), tells
// the peers at the end, and every CTA then waits, on the very barriers those
// writes complete on, until each write sent to it has landed (the bytes no
// peer will send are completed locally); a last cluster barrier then keeps
// every CTA's shared memory alive until no copy reads or writes it any more.
#include <algorithm>
#include <cstring>
#include <string>

#include "ctx.cuh"
#include "sim_device.cuh"
#include "tc_ptx.cuh"

namespace simnet {

struct CArgs {
    CUtensorMap tW[3];   // conv weights [C][K_l] (GEMM layout), box C rows x 128 bytes
    CUtensorMap tF;      // FC1 weights [H][K1], box H/CS rows x 128 bytes
    const float *cbias[3];
    // FP8: per-output-channel weight scales of the conv layers and FC1, and the conv
    // layers' requantisation multipliers (1 / the next layer's input scale)
    const float *cws[3], *cos[3], *fws;
    const float *fbias, *w2, *b2, *fc1_const;
    const StepArgs *A;
    int32_t *status;
    unsigned long long *prof;   // [32] summed SM clock cycles per phase in CTA 0 (or null)
    unsigned long long *tinfo;  // [4] first expired wait: site, CTA, step, pass (zero at launch)
    unsigned long long *pos_sum;  // [2] positions computed and cluster-steps run (accumulated)
    int64_t n_steps, spin_ns;
    int L, C, H, cap, rows_n, stages, stage_bytes;
};

namespace {
using namespace tcx;

// A cluster of CS CTAs (4 or 8) owns 128 batch slots, 128 / CS per CTA.
// Roles: warp 0 TMA producer, warp 1 FC1-done signal, warp 2 MMAs, warps 3-10 workers.
constexpr int kCThreads = 352;
constexpr int kWk = 256;          // worker threads
// One weight stage: consecutive panels (N rows x 64 K-columns BF16, at most 16 KB) of
// one layer, as many as fit in 16 or 32 KB (the larger where three such stages fit);
// one full and one empty barrier per stage, so the MMA thread waits and commits once
// per stage, not once per panel.
constexpr int kPanelMax = 16384;
constexpr int kTmemCols = 512;

__host__ __device__ inline uint32_t al_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Last-conv positions per pass: the first layer's rows of a pass (positions x
// 2^(L-1) pairs x 32 slots) fill at most two 128-row MMA tiles.
__host__ __device__ inline int pass_positions(int L) { return 8 >> (L - 1); }

// Shared-memory layout, offsets from the 1024-byte aligned base.
struct CLay {
    uint32_t ring, act, fc1a, qring, mring, rec, part, prm, slot, misc, bars, total;
};

// FC2 partial sums per (source CTA, column half, slot): 2 floats (regression
// head), 3 padded to 4 (regression head with the store latency), or the hybrid
// head's 22 padded to 24 (16-byte stores).
__host__ __device__ inline int part_floats(int no) { return no == 2 ? 2 : no == 3 ? 4 : 24; }
// prm: conv biases [L*C] | FC1 bias [HN] | S[e] [HN] | b2 [24] | FC2 rows of this
// CTA's neurons: [2][HN] or [3][HN] (regression) or [HN][24] (hybrid, padded) |
// FP8 only: conv weight scales [L*C], conv requantisation [L*C], FC1 weight scales [HN].
__host__ __device__ inline int prm_floats(int L, int C, int HN, int no, int es) {
    return L * C + 2 * HN + 24 + (no == 2 ? 2 * HN : no == 3 ? 3 * HN : 24 * HN) + (es == 1 ? 2 * L * C + HN : 0);
}

// es: bytes per operand element (2 BF16, 1 FP8).  Every operand row is a 128-byte
// swizzled row of 128 / es elements.
__host__ __device__ inline CLay c_layout(int CS, int L, int C, int H, int cap, int stages, int no, int stage_bytes,
                                         int es) {
    CLay y;
    const int HN = H / CS, SPC = 128 / CS, PM = pass_positions(L);
    // operand of layer l: its rows (pass positions x pairs x slots) x K, in 128-byte panels
    uint32_t actb = (uint32_t)(PM * (1 << (L - 1)) * SPC) * 128u * (uint32_t)es;
    for (int l = 1; l < L; l++) {
        const uint32_t b = (uint32_t)(PM * (1 << (L - 1 - l)) * SPC) * 2u * (uint32_t)(es * C);
        actb = b > actb ? b : actb;
    }
    y.ring = 0;
    y.act = (uint32_t)stages * (uint32_t)stage_bytes;
    y.fc1a = al_up(y.act + actb, 1024);
    y.qring = y.fc1a + 128u * (uint32_t)(pass_positions(L) * C * es);      // 128 slots x positions x C
    y.mring = y.qring + (uint32_t)SPC * cap * 8;                            // memory write queues (n_out 3)
    y.rec = y.mring + (no == 3 ? (uint32_t)SPC * cap * 8 : 0u);
    y.part = al_up(y.rec + SPC * 4 * 4, 16);
    y.prm = y.part + 2 * CS * SPC * 4 * part_floats(no);
    y.slot = al_up(y.prm + (uint32_t)prm_floats(L, C, HN, no, es) * 4, 16);
    y.misc = y.slot + SPC * 8 + 10 * SPC * 4;
    // misc: extents in | control words | 32 phase counters (profiling) | exit counters
    // (64 ints) | what every peer sent this CTA (one uint4 per peer)
    y.bars = al_up(y.misc + 16 * CS + 32 + 32 * 8 + 256 + 128, 8);
    y.total = y.bars + (2 * stages + 21) * 8;
    return y;
}

// ------------------------------------------------------------------ cluster PTX
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory offset in CTA `r` of the cluster
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t r) {
    uint32_t o;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(a), "r"(r));
    return o;
}
// Asynchronous stores into CTA r's shared memory (a and bar from mapa): the bytes are
// counted (complete_tx) on the barrier `bar` there; the storing thread does not wait.
__device__ __forceinline__ void cl_st_async_v4(uint32_t a, uint4 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1,%2,%3,%4}, [%5];" ::"r"(a),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cl_st_async_v2(uint32_t a, uint32_t x, uint32_t y, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1,%2}, [%3];" ::"r"(a), "r"(x),
                 "r"(y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool cl_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait that lets the hardware suspend the thread (up to `hint_ns`) until the
// phase completes, so that waiting warps do not take issue slots from working ones.
__device__ __forceinline__ bool try_sleep(uint32_t bar, uint32_t parity, uint32_t hint_ns, bool cluster_scope) {
    uint32_t ok;
    if (cluster_scope)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(hint_ns)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(hint_ns)
            : "memory");
    return ok != 0;
}
// Bounded wait, suspending between polls.
__device__ __noinline__ bool sleep_wait_slow(uint32_t bar, uint32_t parity, int64_t limit, volatile int *abort_flag,
                                             int32_t *status, bool cluster_scope) {
    const uint64_t t0 = gtimer();
    while (true) {
        if (try_sleep(bar, parity, 20000u, cluster_scope)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(gtimer() - t0) > limit) {
            *abort_flag = 1;
            atomicExch(status, kStatusTimeout);
            return false;
        }
    }
}
// Non-blocking test of a phase that other CTAs of the cluster arrive on.
__device__ __forceinline__ bool cl_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a phase of a barrier that other CTAs of the cluster arrive on.
__device__ __noinline__ bool cl_wait_slow(uint32_t bar, uint32_t parity, int64_t limit, volatile int *abort_flag,
                                          int32_t *status) {
    if (cl_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        // suspended until the phase completes (or the hint runs out): no polling that
        // competes with the MMA thread's barrier operations
        if (try_sleep(bar, parity, 20000u, true)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(gtimer() - t0) > limit) {
            *abort_flag = 1;
            atomicExch(status, kStatusTimeout);
            return false;
        }
    }
}
__device__ __forceinline__ bool cl_wait(uint32_t bar, uint32_t parity, int64_t limit, volatile int *abort_flag,
                                        int32_t *status) {
    if (cl_test(bar, parity)) return true;
    return cl_wait_slow(bar, parity, limit, abort_flag, status);
}
__device__ __forceinline__ bool sleep_wait(uint32_t bar, uint32_t parity, int64_t limit, volatile int *abort_flag,
                                           int32_t *status, bool cluster_scope) {
    if (cluster_scope ? cl_test(bar, parity) : mbar_test(bar, parity)) return true;
    return sleep_wait_slow(bar, parity, limit, abort_flag, status, cluster_scope);
}
// Wait for copies or MMAs this CTA started to land, also after an abort (they
// write shared memory or TMEM that is released afterwards); bounded, silent.
__device__ __noinline__ void drain_wait(uint32_t bar, uint32_t parity, int64_t limit) {
    const uint64_t t0 = gtimer();
    while (!cl_try(bar, parity) && (int64_t)(gtimer() - t0) < limit) {
    }
}
// Arrive on a barrier of another CTA of the cluster (shared::cluster address
// from mapa); the release orders this thread's earlier writes before it.
__device__ __forceinline__ void cl_arrive_remote(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
// Complete `bytes` of a local barrier's transaction count: stands in for bytes
// that were expected but that no peer will send.
__device__ __forceinline__ void mbar_complete_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Plain 16-byte store into another CTA's shared memory (made visible by the next
// cluster barrier).
__device__ __forceinline__ void cl_st_v4(uint32_t a, uint4 v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
// 64 consecutive TMEM columns of this warp's 32 lanes (two 32x32b loads, one
// wait, in one statement so that no use of the registers precedes the wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[2][32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
          "=r"(r[0][7]), "=r"(r[0][8]), "=r"(r[0][9]), "=r"(r[0][10]), "=r"(r[0][11]), "=r"(r[0][12]),
          "=r"(r[0][13]), "=r"(r[0][14]), "=r"(r[0][15]), "=r"(r[0][16]), "=r"(r[0][17]), "=r"(r[0][18]),
          "=r"(r[0][19]), "=r"(r[0][20]), "=r"(r[0][21]), "=r"(r[0][22]), "=r"(r[0][23]), "=r"(r[0][24]),
          "=r"(r[0][25]), "=r"(r[0][26]), "=r"(r[0][27]), "=r"(r[0][28]), "=r"(r[0][29]), "=r"(r[0][30]),
          "=r"(r[0][31]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
          "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[1][8]), "=r"(r[1][9]), "=r"(r[1][10]), "=r"(r[1][11]),
          "=r"(r[1][12]), "=r"(r[1][13]), "=r"(r[1][14]), "=r"(r[1][15]), "=r"(r[1][16]), "=r"(r[1][17]),
          "=r"(r[1][18]), "=r"(r[1][19]), "=r"(r[1][20]), "=r"(r[1][21]), "=r"(r[1][22]), "=r"(r[1][23]),
          "=r"(r[1][24]), "=r"(r[1][25]), "=r"(r[1][26]), "=r"(r[1][27]), "=r"(r[1][28]), "=r"(r[1][29]),
          "=r"(r[1][30]), "=r"(r[1][31])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
}
// 16 consecutive TMEM columns of this warp's 32 lanes, waited for.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// 32 or 64 columns from taddr into r[0] (and r[1]).
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, int cols, uint32_t (&r)[2][32]) {
    if (cols > 32) tmem_ld64(taddr, r);
    else tmem_ld32(taddr, r[0]);
}
// 16 TMEM lanes from taddr's lane x 16 columns, waited for: thread t gets lanes t/4 and
// t/4 + 8, columns 2(t%4), 2(t%4) + 1 (r[0..3]) and those columns + 8 (r[4..7]) -- the
// fragment layout of an 8x8 16-bit matrix per register pair (16x256b shape, two repeats).
__device__ __forceinline__ void tmem_ld16x256b_x2(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
}
// Four 8x8 16-bit matrices (fragments f[0..3]) stored transposed: thread 8i + j gives the
// shared-memory address of row j of transposed matrix i (16 contiguous bytes).
__device__ __forceinline__ void stmatrix_x4_trans(uint32_t addr, const uint32_t (&f)[4]) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(f[0]),
                 "r"(f[1]), "r"(f[2]), "r"(f[3])
                 : "memory");
}
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// workers_sync that also returns whether p holds in any worker thread
__device__ __forceinline__ bool workers_any(bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, 1, 256, q;\n selp.u32 %0, 1, 0, o;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from this CTA's
// shared memory into CTA r's, counted (complete_tx) on a barrier in CTA r.
__device__ __forceinline__ void cl_bulk_copy(uint32_t dst_cluster, uint32_t src, uint32_t bytes, uint32_t bar_cluster) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst_cluster),
                 "r"(src), "r"(bytes), "r"(bar_cluster)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }


// Cluster extent from the CTAs' (longest queue + 1, live slots).
template <int CS>
__device__ __forceinline__ void read_ext(const int2 *ext_in, int b, int &E, int &AL) {
    E = 0;
    AL = 0;
    for (int r = 0; r < CS; r++) {
        const volatile int *v = reinterpret_cast<const volatile int *>(&ext_in[b * CS + r]);
        E = max(E, v[0]);
        AL += v[1];
    }
}
__device__ __forceinline__ int positions_of(int E, int L, int rows_n) {
    const int span = 1 << L;
    return max(1, min((E + span - 1) / span, rows_n));
}
// The positions a step computes: at least the first pass, and whole 128-byte FC1
// operand panels (FP8 with 64 channels: positions in pairs; rows_n is then even).
__device__ __forceinline__ int step_positions(int E, int L, int rows_n, int first, int e_round) {
    const int e = max(positions_of(E, L, rows_n), first);
    return min(rows_n, (e + e_round - 1) / e_round * e_round);
}

template <int CS, int NO, bool F8>
__global__ void __launch_bounds__(kCThreads, 1) cluster_kernel(const __grid_constant__ CArgs a) {
    constexpr int SPC = 128 / CS;   // batch slots per CTA
    // operand elements: BF16, or FP8 e4m3 (kind::f8f6f4 MMAs, per-channel scales); a
    // 128-byte swizzled operand row holds EPP of them, one MMA consumes 32 bytes of K
    constexpr int ES = F8 ? 1 : 2, EPP = 128 / ES;
    // positions per 128-byte FC1 operand panel (2 for FP8 with 64 channels): a step
    // computes whole panels, so its extent is rounded up to a multiple of this
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int L = a.L, C = a.C, HN = a.H / CS, S = a.stages, cap = a.cap, PM = pass_positions(L);
    const int kERound = max(1, EPP / C);
    const uint32_t kStage = (uint32_t)a.stage_bytes;
    constexpr bool SQ = NO == 3;            // store latency and memory write queue (Sec. 3.2)
    constexpr int NL = SQ ? 3 : 2;          // latencies per instruction
    constexpr int PF = NO == 2 ? 2 : NO == 3 ? 4 : 24;   // part_floats(NO)
    const CLay y = c_layout(CS, L, C, a.H, cap, S, NO, a.stage_bytes, ES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cl_rank();
    const int slot0 = (int)(blockIdx.x / CS) * 128 + (int)rank * SPC;
    const StepArgs *A = a.A;
    const int64_t lim = a.spin_ns;
    const int64_t drain_ns = lim > 200000000 ? lim : 200000000;   // 0.2 s at least
    // Record where the first expired wait of the launch was (sites: 1 weight stage free,
    // 2 extent (producer), 3 weight panel, 4 (unused), 5 conv layer done, 6 exchange
    // buffer free, 7 exchanged rows in, 8 FC1 done, 9 FC2 partial sums in, 10 FC1 done
    // (warp 1's signal to the cluster), 11 feature rows in, 12 / 13 first / second channel
    // half of a layer's output in, 14 the step's extent published by the producer).
    auto note = [&](bool ok, int site, int64_t step, int64_t pass) -> bool {
        if (!ok && *(volatile int32_t *)a.status == kStatusTimeout &&
            atomicCAS(&a.tinfo[0], 0ull, (unsigned long long)site) == 0ull) {
            a.tinfo[1] = blockIdx.x;
            a.tinfo[2] = (unsigned long long)step;
            a.tinfo[3] = (unsigned long long)pass;
        }
        return ok;
    };

    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + y.bars);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    // 0..S-1 weight panel full, S..2S-1 empty; then:
    // B_FULL + i: the peers' rows of FC1 operand panel i (at most 8 panels a pass)
    // bytes a phase of B_PART / B_EXT receives: every CTA's FC2 partials (two column halves)
    // for this CTA's slots; every CTA's (extent, live count)
    constexpr uint32_t kPartBytes = 2u * CS * SPC * PF * 4u, kExtBytes = CS * 8u;
    const int B_D = 2 * S, B_DFC = 2 * S + 2, B_PART = 2 * S + 3, B_EXT = 2 * S + 4,
              B_FIN = 2 * S + 6, B_FULL = 2 * S + 7, B_F1D = 2 * S + 15;
    // the workers' signals to the MMA warp (one arrival per worker warp, after its writes):
    // a pass's feature rows, the first and the second channel half of a layer's output; and
    // the step's extent (worker thread 0)
    const int B_ROWS = 2 * S + 17, B_HA = 2 * S + 18, B_HB = 2 * S + 19, B_CTL = 2 * S + 20;
    // the exchanged rows of pass R may be overwritten once every CTA's FC1 of pass R is
    // done: CS arrivals on B_EMPTY + (R & 1) (two barriers, so that an arrival for the
    // next pass can never complete the phase of this one)
    auto b_empty = [&](int64_t r) { return bar((r & 1) ? 2 * S + 16 : 2 * S + 1); };
    // The FC1 operand is exchanged in units: its 128-byte panels (one CTA's rows of one:
    // SPC x 128 bytes), or, for FP8 with 128 channels (a panel is one position), half panels
    // of 64-byte rows with 64-byte swizzle, one per position and channel half, so that the
    // first channel half travels while the second is converted.
    const bool hfc = F8 && C == 128;
    const uint32_t xbytes = hfc ? (uint32_t)SPC * 64u : (uint32_t)SPC * 128u;   // one CTA's rows of a unit
    const uint32_t xstride = hfc ? 8192u : 16384u;                             // between units
    auto xunits = [&](int P) { return hfc ? 2 * P : P * C / EPP; };
    float *s_cb = reinterpret_cast<float *>(sm + y.prm);   // [L][C] conv biases
    float *s_fb = s_cb + L * C;                              // [HN] FC1 bias of this CTA's neurons
    float *s_Se = s_fb + HN;                                 // [HN] S[e] of the current step (+ FC1 bias)
    float *s_b2 = s_Se + HN;                                 // [24] FC2 bias
    float *s_w2 = s_b2 + 24;                                 // FC2 rows for this CTA's neurons
    float *s_w2f = s_w2, *s_w2e = s_w2 + HN;                 // regression: [2][HN]; hybrid: [HN][24]
    float *s_ws = s_w2 + (NO == 2 ? 2 * HN : NO == 3 ? 3 * HN : 24 * HN);   // FP8: [L][C] weight scales
    float *s_os = s_ws + L * C;                                  // FP8: [L][C] requantisation (folded into s_ws, s_cb)
    float *s_fws = s_os + L * C;                                 // FP8: [HN] FC1 weight scales
    int64_t *s_o = reinterpret_cast<int64_t *>(sm + y.slot);
    int32_t *s_b = reinterpret_cast<int32_t *>(s_o + SPC), *s_n = s_b + SPC, *s_p = s_n + SPC,
            *s_tick = s_p + SPC, *s_qs = s_tick + SPC, *s_ql = s_qs + SPC, *s_ev = s_ql + SPC,
            *s_al = s_ev + SPC, *s_ms = s_al + SPC, *s_ml = s_ms + SPC;   // s_ms/s_ml: write queue
    uint64_t *qring = reinterpret_cast<uint64_t *>(sm + y.qring);
    uint64_t *mring = reinterpret_cast<uint64_t *>(sm + y.mring);   // used with SQ only
    uint32_t *recb = reinterpret_cast<uint32_t *>(sm + y.rec);   // [slot][position & 3]
    float *part = reinterpret_cast<float *>(sm + y.part);       // [source CTA * 2 + half][slot][PF]
    int2 *ext_in = reinterpret_cast<int2 *>(sm + y.misc);       // [step parity][source CTA]
    volatile int *ctl = reinterpret_cast<volatile int *>(sm + y.misc + 16 * CS);   // positions, stop
    volatile int *abort_f = ctl + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + y.misc + 16 * CS + 20);
    int *cnt = reinterpret_cast<int *>(sm + y.misc + 16 * CS + 24);   // weight panels issued, consumed
    // phase counters (CTA 0, on request): shared-memory accumulators, written out at the end
    unsigned long long *pacc = reinterpret_cast<unsigned long long *>(sm + y.misc + 16 * CS + 32);
    // exit counters: what this CTA sent (X_*_SENT), consumed (X_*_CONS, X_ROWS_DONE) and armed
    volatile int *xs = reinterpret_cast<volatile int *>(sm + y.misc + 16 * CS + 32 + 256);
    enum { X_EXT_SENT = 0, X_PART_SENT, X_EXT_CONS, X_PART_CONS, X_ROWS_DONE, X_FC1_WAITED, X_ARMED_R, X_ARMED_NP,
           X_FPH, X_DONE, X_F1C, X_ROWS_SENT = 16, X_ROWS_NP = 24 };
    uint4 *inbox = reinterpret_cast<uint4 *>(sm + y.misc + 16 * CS + 32 + 512);   // [source CTA]

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(bar(s), 1);
            mbar_init(bar(S + s), 1);    // free once this CTA's MMAs have read it
        }
        mbar_init(bar(B_D), 1);
        for (int i = 0; i < 8; i++) mbar_init(bar(B_FULL + i), 1);   // thread 0's expect_tx; the peers' copies
        mbar_init(b_empty(0), CS);
        mbar_init(b_empty(1), CS);
        mbar_init(bar(B_DFC), 1);
        // partial sums and extents arrive by st.async, counted in bytes: one local
        // arrival (with the byte count) per phase, made here for the first phases
        mbar_init(bar(B_PART), 1);
        mbar_init(bar(B_EXT), 1);
        mbar_init(bar(B_EXT + 1), 1);
        mbar_expect_tx(bar(B_PART), kPartBytes);
        mbar_expect_tx(bar(B_EXT), kExtBytes);
        mbar_expect_tx(bar(B_EXT + 1), kExtBytes);
        mbar_init(bar(B_FIN), 1);
        mbar_init(bar(B_F1D), 1);
        mbar_init(bar(B_ROWS), 8);
        mbar_init(bar(B_HA), 8);
        mbar_init(bar(B_HB), 8);
        mbar_init(bar(B_CTL), 1);
        *abort_f = 0;
        cnt[0] = cnt[1] = 0;
        for (int k = 0; k < 32; k++) pacc[k] = 0;
        for (int k = 0; k < 64; k++) xs[k] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // constants of this CTA's share
    for (int i = threadIdx.x; i < L * C; i += blockDim.x) {
        s_cb[i] = a.cbias[i / C][i % C];
        if constexpr (F8) {
            // the requantisation multiplier (1 / the next layer's input scale, positive)
            // folded in: ReLU(acc w + b) m = ReLU(acc (w m) + b m)
            const float m = a.cos[i / C][i % C];
            s_ws[i] = a.cws[i / C][i % C] * m;
            s_cb[i] *= m;
            s_os[i] = m;
        }
    }
    for (int j = threadIdx.x; j < HN; j += blockDim.x) {
        const int nn = (int)rank * HN + j;
        s_fb[j] = a.fbias[nn];
        if constexpr (F8) s_fws[j] = a.fws[nn];
        if constexpr (NO == 2 || NO == 3) {
            s_w2f[j] = a.w2[nn];
            s_w2e[j] = a.w2[a.H + nn];
            if constexpr (SQ) s_w2f[2 * HN + j] = a.w2[2 * a.H + nn];
        }
    }
    if constexpr (NO != 2 && NO != 3)
        for (int i = threadIdx.x; i < HN * 24; i += blockDim.x) {
            const int j = i / 24, o = i % 24;
            s_w2[i] = o < NO ? a.w2[(size_t)o * a.H + (int)rank * HN + j] : 0.f;
        }
    if (threadIdx.x < 24) s_b2[threadIdx.x] = threadIdx.x < NO ? a.b2[threadIdx.x] : 0.f;
    // slot state (workers: warp w takes slots w-3, w+5, ...)
    if (warp >= 3) {
        const int n_act = min(*A->n_active, A->n_sub);
        for (int j = 0; j < SPC / 8; j++) {
            const int s = (warp - 3) + 8 * j, g = slot0 + s;
            int b = -1;
            int64_t o = 0;
            int n = 0, p = 0;
            if (g < n_act) {
                b = A->active[g];
                o = A->offsets[b];
                n = (int)(A->offsets[b + 1] - o);
                p = A->pos[b];
                for (int i = lane; i < cap; i += 32) qring[s * cap + i] = A->ring[(size_t)b * cap + i];
                if constexpr (SQ)
                    for (int i = lane; i < cap; i += 32) mring[s * cap + i] = A->mring[(size_t)b * cap + i];
            }
            if (lane == 0) {
                s_b[s] = b;
                s_o[s] = o;
                s_n[s] = n;
                s_p[s] = p;
                s_tick[s] = b >= 0 ? A->tick[b] : 0;
                s_qs[s] = b >= 0 ? A->qstart[b] : 0;
                s_ql[s] = b >= 0 ? A->qlen[b] : 0;
                s_ev[s] = b >= 0 ? A->evict[b] : 0;
                s_al[s] = (b >= 0 && p < n) ? 1 : 0;
                s_ms[s] = (SQ && b >= 0) ? A->mstart[b] : 0;
                s_ml[s] = (SQ && b >= 0) ? A->mlen[b] : 0;
                if (p < n) recb[s * 4 + (p & 3)] = A->records[o + p];
                if (p + 1 < n) recb[s * 4 + ((p + 1) & 3)] = A->records[o + p + 1];
            }
        }
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    cluster_sync_all();   // every CTA's barriers are initialised before anyone arrives remotely

    const uint32_t ring0 = smem_u32(sm + y.ring), act0 = smem_u32(sm + y.act), fc0 = smem_u32(sm + y.fc1a);
    // TMEM columns: layer 0 tiles at 0 (two tiles of C), odd layers at 256, even layers >= 2 at 0, FC1 at 384
    auto dcol = [&](int l) -> uint32_t { return l == 0 ? 0u : ((l & 1) ? 256u : 0u); };
    auto rows_of = [&](int l, int P) { return P * (1 << (L - 1 - l)) * SPC; };    // layer l's A rows
    auto tiles_of = [&](int l, int P) { return (rows_of(l, P) + 127) / 128; };
    // bytes between the 64-column K panels of layer l's operand: the panels hold just the
    // pass's rows; an MMA tile past them reads neighbouring shared memory into rows it ignores
    auto pstride_of = [&](int l, int P) { return (uint32_t)rows_of(l, P) * 128u; };
    auto panels_of = [&](int l) { return l == 0 ? 128 / EPP : 2 * C / EPP; };   // K / EPP
    // panels a stage holds: conv panels are C x 64, FC1 panels HN x 64 (BF16)
    const int kConvPer = (int)kStage / (C * 128), kFcPer = min((int)kStage / (HN * 128), 8);
    auto conv_stages = [&](int l) { return (panels_of(l) + kConvPer - 1) / kConvPer; };
    // Channel halves of an operand whose K runs over blocks of C channels (a conv layer's two
    // input rows, or FC1's positions).  With panels of EPP <= C elements the K-steps of half h
    // in a panel are one contiguous run: all or none of a panel half a row wide (BF16,
    // C = 128: the even panels hold the first half), else its first or its last two of four.
    // FP8 with 64 channels (two rows to a panel) is not split.
    const bool kSplit = EPP <= C;
    // load order of layer l's weight panels (l >= 1): the first channel half's panels first
    // where a panel is narrower than a row
    auto conv_perm = [&](int l, int i) -> int {
        if (l == 0 || !(EPP < C)) return i;
        const int hp = panels_of(l) / 2;
        return i < hp ? 2 * i : 2 * (i - hp) + 1;
    };
    // A layer after the first with at most 64 rows in the pass (BF16, 128 channels) runs with
    // the operands swapped: the weights as the 128-row side (M = output channels), the pass's
    // rows as N.  An MMA's time follows N (measured: N = 128, 64, 32 take ~73, ~57, ~48
    // cycles; M = 64 saves nothing), and every worker warp then has output channels to
    // convert (TMEM lanes = channels).
    auto swapped = [&](int l, int P) { return !F8 && C == 128 && l >= 1 && rows_of(l, P) <= 64; };
    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int it = 0, ps = 0;     // panels issued; stage of the next one
            uint32_t pph = 0;       // and its phase parity (no division on the issue path)
            auto adv = [&] {
                it++;
                if (++ps == S) { ps = 0; pph ^= 1u; }
            };
            bool ok = true;
            // n panels of pb bytes (K-columns x0, x0 + xs, ...) into the next stage: whole
            // conv panels (all C rows) or this CTA's rows of FC1 panels
            auto load = [&](const CUtensorMap *m, int x0, int xs, int yy, uint32_t pb, int n) {
                const int s = ps;
                if (!note(mbar_wait(bar(S + s), pph ^ 1u, lim, abort_f, a.status), 1, -1, it)) {
                    ok = false;
                    return;
                }
                mbar_expect_tx(bar(s), (uint32_t)n * pb);
                for (int j = 0; j < n; j++)
                    tma_load_2d(ring0 + (uint32_t)s * kStage + (uint32_t)j * pb, m, bar(s), x0 + xs * j, yy);
                adv();
            };
            // conv stage i of a pass (all layers' weights in consumption order), i in [from, to)
            int n_conv_stages = 0;
            for (int l = 0; l < L; l++) n_conv_stages += conv_stages(l);
            auto conv_loads = [&](int from, int to) {
                int i = 0;
                for (int l = 0; l < L && ok; l++)
                    for (int g = 0; g < conv_stages(l) && ok; g++, i++) {
                        if (i < from || i >= to) continue;
                        const int p0 = g * kConvPer, n = min(kConvPer, panels_of(l) - p0);
                        // panels in the MMA warp's order (a stage's panels are evenly spaced)
                        const int x0 = conv_perm(l, p0) * EPP, xs = n > 1 ? (conv_perm(l, p0 + 1) - conv_perm(l, p0)) * EPP : 0;
                        load(&a.tW[l], x0, xs, 0, (uint32_t)C * 128u, n);
                    }
            };
            // Before a step's extent is known only its first S stages are loaded: they are
            // freed by the current step, which every CTA finishes; a stage holding one of
            // those panels is freed only if the step runs (the cluster may be done by then).
            const int pre = min(n_conv_stages, S);
            if (a.n_steps > 0) conv_loads(0, pre);
            for (int64_t t = 0; t < a.n_steps && ok; t++) {
                // The step's extent (the cluster's longest context + 1, and its live count),
                // published to the MMA warp and the workers through ctl (double-buffered by
                // step): neither waits for the cluster's slowest head before its first layer.
                const bool w = note(cl_wait(bar(B_EXT + (int)(t & 1)), (uint32_t)(t >> 1) & 1u, lim, abort_f, a.status), 2, t, 0);
                int E = 0, AL = 0;
                if (w) {
                    read_ext<CS>(ext_in, (int)(t & 1), E, AL);
                    mbar_expect_tx(bar(B_EXT + (int)(t & 1)), kExtBytes);   // its phase two steps on
                    xs[X_EXT_CONS] = xs[X_EXT_CONS] + 1;
                }
                const int eL = step_positions(E, L, a.rows_n, min(PM, a.rows_n), kERound);
                volatile int *c = ctl + 2 * (int)(t & 1);
                c[0] = eL;
                c[1] = (!w || AL == 0 || *abort_f) ? 1 : 0;
                mbar_arrive(bar(B_CTL));
                if (c[1]) break;
                for (int q0 = 0; q0 < eL && ok; q0 += PM) {
                    const int P = min(PM, eL - q0);
                    conv_loads(q0 > 0 ? 0 : pre, n_conv_stages);
                    const int np = P * C / EPP;
                    for (int p0 = 0; p0 < np && ok; p0 += kFcPer)
                        load(&a.tF, q0 * C + p0 * EPP, EPP, (int)rank * HN, (uint32_t)HN * 128u, min(kFcPer, np - p0));
                }
                if (t + 1 < a.n_steps) conv_loads(0, pre);   // the next step's first stages
            }
            cnt[0] = it;
        }
    } else if (warp == 2) {
        // ---------------------------------------------------------------- MMA warp
        // The whole warp runs the issue loops (warp-uniform operands, one elected lane issues
        // each MMA) and follows the workers through the step: the first layer's MMAs as soon
        // as the pass's feature rows are in (the first pass's before the cluster's extent is
        // known), then per layer the K-steps of the first channel half of the operand while
        // the workers still write the second half.
        int it = 0, cs = 0;        // weight stages consumed; ring slot of the next one and its phase
        uint32_t cph = 0;
        uint32_t fph = 0;          // phase parity of each B_FULL + i
        uint32_t ph_rows = 0, ph_ha = 0, ph_hb = 0, ph_ctl = 0;   // phases of the workers' signals
        int64_t R = 0;             // passes exchanged
        bool ok = true;
        const bool prof = a.prof && blockIdx.x == 0 && lane == 0;
        // a worker signal (B_ROWS, B_HA, B_HB, B_CTL); the wait's time goes to counter pc
        auto wait_sig = [&](int b, uint32_t &ph, int site, int64_t t, int pc) -> bool {
            const uint64_t t0 = prof ? (uint64_t)clock64() : 0;
            const bool w = note(sleep_wait(bar(b), ph, lim, abort_f, a.status, false), site, t, R);
            ph ^= 1u;
            if (prof) pacc[pc] += (uint64_t)clock64() - t0;
            const bool all = __all_sync(0xffffffffu, w);
            tc_fence_after();
            return all;
        };
        auto take = [&](int &s, int who) -> bool {   // the next weight stage (who: layer, L = FC1)
            s = cs;
            const uint64_t tw = prof ? (uint64_t)clock64() : 0;
            const bool w = note(mbar_wait(bar(s), cph, lim, abort_f, a.status), 3, -1, it);
            if (!__all_sync(0xffffffffu, w)) return false;
            if (prof) pacc[26 + who] += (uint64_t)clock64() - tw;
            tc_fence_after();
            it++;
            if (++cs == S) { cs = 0; cph ^= 1u; }
            return true;
        };
        // K-steps k0 .. k0 + nk - 1 (nk 2 or 4) of one 128-byte operand panel; the layer's
        // first MMA (fresh) overwrites the accumulator
        auto mma_ks = [&](uint32_t d, uint32_t alo, uint32_t blo, uint32_t ID, int k0, int nk, bool &fresh) {
            alo += 2u * (uint32_t)k0;
            blo += 2u * (uint32_t)k0;
            umma_lo<F8>(d, alo, blo, ID, fresh ? 0u : 1u);
            fresh = false;
            umma_lo<F8>(d, alo + 2u, blo + 2u, ID, 1u);
            if (nk == 4) {
                umma_lo<F8>(d, alo + 4u, blo + 4u, ID, 1u);
                umma_lo<F8>(d, alo + 6u, blo + 6u, ID, 1u);
            }
        };
        // Straight-line issue of the K-steps of one or two panels: loops with run-time trip
        // counts between the MMAs cost this warp more than the MMAs themselves take.
        auto mma2 = [&](uint32_t d, uint32_t alo, uint32_t blo, uint32_t ID, uint32_t acc0) {
            umma_lo<F8>(d, alo, blo, ID, acc0);
            umma_lo<F8>(d, alo + 2u, blo + 2u, ID, 1u);
        };
        auto mma4 = [&](uint32_t d, uint32_t alo, uint32_t blo, uint32_t ID, uint32_t acc0) {
            mma2(d, alo, blo, ID, acc0);
            mma2(d, alo + 4u, blo + 4u, ID, 1u);
        };
        const uint32_t act_lo = sdesc_lo(act0), ring_lo = sdesc_lo(ring0), fc_lo = sdesc_lo(fc0);
        const uint32_t cstep = (uint32_t)(C * 128) >> 4, hstep = (uint32_t)(HN * 128) >> 4;
        // the first layer over a pass's rows (all K-steps: the rows are built whole)
        auto conv_first = [&](int P) -> bool {
            const int T = tiles_of(0, P), np = panels_of(0), G = conv_stages(0);
            const uint32_t ID = idesc_rt(C, F8), astep = pstride_of(0, P) >> 4;
            bool f0 = true, f1 = true;
            if (G == 1 && T == 1 && np <= 2) {   // one stage, one tile (c2's shapes): straight line
                int s;
                if (!take(s, 0)) return false;
                const uint32_t b0 = ring_lo + ((uint32_t)s * kStage >> 4);
                mma4(tmem_base, act_lo, b0, ID, 0u);
                if (np == 2) mma4(tmem_base, act_lo + astep, b0 + cstep, ID, 1u);
                umma_commit_warp(bar(S + s));
                umma_commit_warp(bar(B_D));
                return true;
            }
            for (int g = 0; g < G; g++) {
                int s;
                if (!take(s, 0)) return false;
                const int n = min(kConvPer, np - g * kConvPer);
                for (int j = 0; j < n; j++) {
                    const int pi = g * kConvPer + j;
                    const uint32_t a0 = act_lo + (uint32_t)pi * astep, b0 = ring_lo + ((uint32_t)s * kStage >> 4) + (uint32_t)j * cstep;
                    mma_ks(tmem_base, a0, b0, ID, 0, 4, f0);
                    if (T == 2) mma_ks(tmem_base + (uint32_t)C, a0 + 1024u, b0, ID, 0, 4, f1);
                }
                umma_commit_warp(bar(S + s));   // the stage is free once these MMAs have read it
            }
            umma_commit_warp(bar(B_D));
            return true;
        };
        // Layer l >= 1 (one 128-row tile): its operand's channel halves as the workers finish
        // them.  The issue path carries as little arithmetic as possible (the MMA warp shares
        // its scheduler with two busy worker warps while it issues the first half).
        auto conv_next = [&](int l, int P, int64_t t) -> bool {
            const int np = panels_of(l), G = conv_stages(l);
            const uint32_t ID = idesc_rt(C, F8), astep = pstride_of(l, P) >> 4, d = tmem_base + dcol(l);
            bool fresh = true;
            if (!kSplit) {   // FP8 with 64 channels: everything once both halves are in
                if (!wait_sig(B_HA, ph_ha, 12, t, 20 + l) || !wait_sig(B_HB, ph_hb, 13, t, 20 + l)) return false;
                const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                for (int g = 0; g < G; g++) {
                    int s;
                    if (!take(s, l)) return false;
                    const int n = min(kConvPer, np - g * kConvPer);
                    const uint32_t b0 = ring_lo + ((uint32_t)s * kStage >> 4);
                    for (int j = 0; j < n; j++)
                        mma_ks(d, act_lo + (uint32_t)(g * kConvPer + j) * astep, b0 + (uint32_t)j * cstep, ID, 0, 4, fresh);
                    umma_commit_warp(bar(S + s));
                }
                if (prof) pacc[23 + l] += (uint64_t)clock64() - ti;
            } else if (EPP < C && kConvPer == 2 && np == 4) {
                // BF16, 128 channels, 32 KB stages (c2): per half one stage of panels h, 2 + h
                const bool sw = swapped(l, P);
                const uint32_t IDs = sw ? idesc_rt(rows_of(l, P), false) : ID;
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20 + l)) return false;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    int s;
                    if (!take(s, l)) return false;
                    const uint32_t b0 = ring_lo + ((uint32_t)s * kStage >> 4), a0 = act_lo + (uint32_t)h * astep;
                    if (sw) {   // weights as A (M = channels), the pass's rows as B
                        mma4(d, b0, a0, IDs, h ? 1u : 0u);
                        mma4(d, b0 + cstep, a0 + 2u * astep, IDs, 1u);
                    } else {
                        mma4(d, a0, b0, ID, h ? 1u : 0u);
                        mma4(d, a0 + 2u * astep, b0 + cstep, ID, 1u);
                    }
                    umma_commit_warp(bar(S + s));
                    if (prof) pacc[23 + l] += (uint64_t)clock64() - ti;
                }
            } else if (EPP == C && G == 1 && np == 2) {
                // one stage of two row-wide panels (FP8 with 128 channels, BF16 with 64): K-steps
                // 0-1 of both panels for the first half, 2-3 for the second
                int s = 0;
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20 + l)) return false;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    if (h == 0 && !take(s, l)) return false;
                    const uint32_t b0 = ring_lo + ((uint32_t)s * kStage >> 4) + 4u * (uint32_t)h, a0 = act_lo + 4u * (uint32_t)h;
                    mma2(d, a0, b0, ID, h ? 1u : 0u);
                    mma2(d, a0 + astep, b0 + cstep, ID, 1u);
                    if (h == 1) umma_commit_warp(bar(S + s));
                    if (prof) pacc[23 + l] += (uint64_t)clock64() - ti;
                }
            } else if (EPP < C) {
                // panels half a row wide (BF16, 128 channels): the stages of the first half hold
                // the even panels (rows 2j, 2j+1, channels 0-63), those of the second the odd ones
                const int hp = np / 2, Gh = G / 2;
                const bool sw = swapped(l, P);
                const uint32_t IDs = sw ? idesc_rt(rows_of(l, P), false) : ID;
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20 + l)) return false;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    for (int g = 0; g < Gh; g++) {
                        int s;
                        if (!take(s, l)) return false;
                        const int i0 = g * kConvPer, n = min(kConvPer, hp - i0);
                        const uint32_t b0 = ring_lo + ((uint32_t)s * kStage >> 4);
                        uint32_t a = act_lo + (uint32_t)(2 * i0 + h) * astep;
                        for (int j = 0; j < n; j++, a += 2u * astep) {
                            if (sw) mma_ks(d, b0 + (uint32_t)j * cstep, a, IDs, 0, 4, fresh);
                            else mma_ks(d, a, b0 + (uint32_t)j * cstep, ID, 0, 4, fresh);
                        }
                        umma_commit_warp(bar(S + s));
                    }
                    if (prof) pacc[23 + l] += (uint64_t)clock64() - ti;
                }
            } else {
                // panels a row wide (BF16 with 64 channels, FP8 with 128): K-steps 0-1 of every
                // panel are the first half, 2-3 the second; the layer's stages (at most two)
                // stay held until the second half is issued
                int s0 = 0, s1 = 0;
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20 + l)) return false;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    for (int g = 0; g < G; g++) {
                        if (h == 0) {
                            int s;
                            if (!take(s, l)) return false;
                            if (g == 0) s0 = s; else s1 = s;
                        }
                        const uint32_t s = g == 0 ? (uint32_t)s0 : (uint32_t)s1;
                        const int n = min(kConvPer, np - g * kConvPer);
                        const uint32_t b0 = ring_lo + (s * kStage >> 4);
                        for (int j = 0; j < n; j++)
                            mma_ks(d, act_lo + (uint32_t)(g * kConvPer + j) * astep, b0 + (uint32_t)j * cstep, ID, 2 * h, 2, fresh);
                        if (h == 1) umma_commit_warp(bar(S + (int)s));
                    }
                    if (prof) pacc[23 + l] += (uint64_t)clock64() - ti;
                }
            }
            umma_commit_warp(bar(B_D));
            return true;
        };
        // FC1 over a pass's positions: per panel once every CTA's rows of it are in; with the
        // split (every FC1 stage of the pass held at once) the first channel half's K-steps first
        auto fc1 = [&](int q0, int P, int64_t t) -> bool {
            const int np = P * C / EPP, G = (np + kFcPer - 1) / kFcPer;   // weight panels (positions for FP8)
            const bool split = kSplit && G <= S;
            const int fmask = kFcPer - 1, fshift = __ffs(kFcPer) - 1;   // kFcPer is a power of two
            const uint32_t ID = idesc_rt(HN, F8), d = tmem_base + 384u;
            bool fresh = q0 == 0;   // FC1 accumulates over the passes
            uint64_t slots = 0;     // ring slot of each stage taken (up to eight)
            int taken = 0;
            // panel pi: its stage (taken at first use), the peers' rows (waited at first use)
            auto panel = [&](int pi, int k0, int nk) -> bool {
                const int g = pi >> fshift, j = pi & fmask;
                while (taken <= g) {
                    int s;
                    if (!take(s, L)) return false;
                    slots |= (uint64_t)s << (8 * taken);
                    taken++;
                }
                if (k0 == 0) {   // first use of the panel
                    const uint64_t tf = prof ? (uint64_t)clock64() : 0;
                    const bool in = note(cl_wait(bar(B_FULL + pi), (fph >> pi) & 1u, lim, abort_f, a.status), 7, t, R);
                    if (!__all_sync(0xffffffffu, in)) return false;
                    fph ^= 1u << pi;
                    if (lane == 0) {
                        xs[X_FPH] = (int)fph;
                        xs[X_FC1_WAITED] = xs[X_FC1_WAITED] | (1 << pi);
                    }
                    if (prof) pacc[18] += (uint64_t)clock64() - tf;
                }
                const uint32_t s = (uint32_t)(slots >> (8 * g)) & 0xffu;
                mma_ks(d, fc_lo + (uint32_t)pi * 1024u, ring_lo + (s * kStage >> 4) + (uint32_t)j * hstep, ID, k0, nk,
                       fresh);
                return true;
            };
            // exchange unit u: the peers' rows of it are in
            auto unit_in = [&](int u) -> bool {
                const uint64_t tf = prof ? (uint64_t)clock64() : 0;
                const bool in = note(cl_wait(bar(B_FULL + u), (fph >> u) & 1u, lim, abort_f, a.status), 7, t, R);
                if (!__all_sync(0xffffffffu, in)) return false;
                fph ^= 1u << u;
                if (lane == 0) {
                    xs[X_FPH] = (int)fph;
                    xs[X_FC1_WAITED] = xs[X_FC1_WAITED] | (1 << u);
                }
                if (prof) pacc[18] += (uint64_t)clock64() - tf;
                return true;
            };
            if (G == 1 && P == 2 && (hfc || (split && EPP < C && np == 4))) {
                // c2's shapes, one weight stage, straight line: per channel half the two units of
                // that half (BF16: panels h and 2 + h; FP8: half panels h and 2 + h against
                // K-steps 2h, 2h + 1 of weight panels 0 and 1)
                int s = 0;
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20)) return false;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    if (h == 0 && !take(s, L)) return false;
                    const uint32_t b0 = ring_lo + ((uint32_t)s * kStage >> 4);
                    const uint32_t acc0 = (h == 0 && fresh) ? 0u : 1u;
                    if (hfc) {
                        if (!unit_in(h)) return false;
                        umma_lo_a<F8>(d, fc_lo + 512u * (uint32_t)h, kSdescHi64, b0 + 4u * (uint32_t)h, ID, acc0);
                        umma_lo_a<F8>(d, fc_lo + 512u * (uint32_t)h + 2u, kSdescHi64, b0 + 4u * (uint32_t)h + 2u, ID, 1u);
                        if (!unit_in(2 + h)) return false;
                        const uint32_t a1 = fc_lo + 512u * (uint32_t)(2 + h), b1 = b0 + hstep + 4u * (uint32_t)h;
                        umma_lo_a<F8>(d, a1, kSdescHi64, b1, ID, 1u);
                        umma_lo_a<F8>(d, a1 + 2u, kSdescHi64, b1 + 2u, ID, 1u);
                    } else {
                        if (!unit_in(h)) return false;
                        mma4(d, fc_lo + 1024u * (uint32_t)h, b0 + (uint32_t)h * hstep, ID, acc0);
                        if (!unit_in(2 + h)) return false;
                        mma4(d, fc_lo + 1024u * (uint32_t)(2 + h), b0 + (uint32_t)(2 + h) * hstep, ID, 1u);
                    }
                    if (prof) pacc[19] += (uint64_t)clock64() - ti;
                }
                umma_commit_warp(bar(S + s));
            } else if (hfc) {
                // FP8, 128 channels: half panel 2 pi + h (64-byte rows) against K-steps 2h, 2h + 1
                // of weight panel pi
                auto hpanel = [&](int pi, int h) -> bool {
                    const int g = pi >> fshift, j = pi & fmask, u = 2 * pi + h;
                    while (taken <= g) {
                        int s;
                        if (!take(s, L)) return false;
                        slots |= (uint64_t)s << (8 * taken);
                        taken++;
                    }
                    const uint64_t tf = prof ? (uint64_t)clock64() : 0;
                    const bool in = note(cl_wait(bar(B_FULL + u), (fph >> u) & 1u, lim, abort_f, a.status), 7, t, R);
                    if (!__all_sync(0xffffffffu, in)) return false;
                    fph ^= 1u << u;
                    if (lane == 0) {
                        xs[X_FPH] = (int)fph;
                        xs[X_FC1_WAITED] = xs[X_FC1_WAITED] | (1 << u);
                    }
                    if (prof) pacc[18] += (uint64_t)clock64() - tf;
                    const uint32_t s = (uint32_t)(slots >> (8 * g)) & 0xffu;
                    const uint32_t alo = fc_lo + (uint32_t)u * 512u, blo = ring_lo + (s * kStage >> 4) + (uint32_t)j * hstep + 4u * (uint32_t)h;
                    umma_lo_a<F8>(d, alo, kSdescHi64, blo, ID, fresh ? 0u : 1u);
                    fresh = false;
                    umma_lo_a<F8>(d, alo + 2u, kSdescHi64, blo + 2u, ID, 1u);
                    return true;
                };
                const bool hold = G <= S;   // every stage held until the second half, else both halves at once
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20)) return false;
                    if (!hold && h == 0) continue;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    for (int pi = 0; pi < P; pi++) {
                        if (hold) {
                            if (!hpanel(pi, h)) return false;
                        } else {
                            if (!hpanel(pi, 0) || !hpanel(pi, 1)) return false;
                            if (pi + 1 == P || ((pi + 1) & fmask) == 0)
                                umma_commit_warp(bar(S + (int)((slots >> (8 * (pi >> fshift))) & 0xffu)));
                        }
                    }
                    if (prof) pacc[19] += (uint64_t)clock64() - ti;
                }
                if (hold)
                    for (int g = 0; g < taken; g++) umma_commit_warp(bar(S + (int)((slots >> (8 * g)) & 0xffu)));
            } else if (!split) {
                if (!wait_sig(B_HA, ph_ha, 12, t, 20) || !wait_sig(B_HB, ph_hb, 13, t, 20)) return false;
                const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                for (int pi = 0; pi < np; pi++) {
                    if (!panel(pi, 0, 4)) return false;
                    if (pi + 1 == np || ((pi + 1) & fmask) == 0)   // the stage's last panel
                        umma_commit_warp(bar(S + (int)((slots >> (8 * (pi >> fshift))) & 0xffu)));
                }
                if (prof) pacc[19] += (uint64_t)clock64() - ti;
            } else {
                for (int h = 0; h < 2; h++) {
                    if (!wait_sig(h ? B_HB : B_HA, h ? ph_hb : ph_ha, h ? 13 : 12, t, 20)) return false;
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    if (EPP < C) {   // the even panels are the first half, the odd ones the second
                        for (int pi = h; pi < np; pi += 2)
                            if (!panel(pi, 0, 4)) return false;
                    } else {         // K-steps 0-1 of every panel, then 2-3
                        for (int pi = 0; pi < np; pi++)
                            if (!panel(pi, 2 * h, 2)) return false;
                    }
                    if (prof) pacc[19] += (uint64_t)clock64() - ti;
                }
                for (int g = 0; g < taken; g++) umma_commit_warp(bar(S + (int)((slots >> (8 * g)) & 0xffu)));
            }
            umma_commit_warp(bar(B_F1D));   // warp 1 tells every CTA once these MMAs are done
            if (lane == 0) {
                xs[X_F1C] = xs[X_F1C] + 1;
                xs[X_ROWS_DONE] = (int)R + 1;
                xs[X_FC1_WAITED] = 0;
            }
            R++;
            return true;
        };
        auto arm_rows = [&](int P) {   // lane 0: the peers' rows of pass R, all panels
            for (int i = 0; i < xunits(P); i++) mbar_expect_tx(bar(B_FULL + i), (uint32_t)(CS - 1) * xbytes);
            xs[X_ARMED_R] = (int)R + 1;
            xs[X_ARMED_NP] = xunits(P);
        };
        const int P0 = min(PM, a.rows_n);
        for (int64_t t = 0; t < a.n_steps && ok; t++) {
            int eL = P0;
            for (int q0 = 0; q0 < eL && ok; q0 += PM) {
                const int P = min(PM, eL - q0);   // P0 for the first pass
                ok = wait_sig(B_ROWS, ph_rows, 11, t, 16);
                if (ok) {
                    const uint64_t ti = prof ? (uint64_t)clock64() : 0;
                    tc_fence_after();
                    ok = conv_first(P);
                    if (prof) pacc[23] += (uint64_t)clock64() - ti;
                }
                // the peers' rows of this pass, expected while its MMAs run (every phase of
                // the previous pass completed before that pass's FC1 MMAs)
                if (ok && lane == 0) arm_rows(P);
                __syncwarp();
                if (ok && q0 == 0) {   // the step's extent: positions, or the cluster is done
                    ok = wait_sig(B_CTL, ph_ctl, 14, t, 17);
                    const volatile int *c = ctl + 2 * (int)(t & 1);
                    if (!ok || c[1]) { ok = false; break; }
                    eL = c[0];
                }
                for (int l = 1; l < L && ok; l++) ok = conv_next(l, P, t);
                if (ok) ok = fc1(q0, P, t);
            }
            if (ok) umma_commit_warp(bar(B_DFC));
        }
        // every MMA done before TMEM is released
        if (lane == 0) {
            cnt[1] = it;
            __threadfence_block();
            xs[X_DONE] = 1;   // no more FC1 commits: warp 1 stops once it has signalled them all
        }
        umma_commit_warp(bar(B_FIN));
        if (lane == 0) drain_wait(bar(B_FIN), 0u, drain_ns);
        __syncwarp();
    } else if (warp >= 3) {
        // ---------------------------------------------------------------- workers
        const int wi = warp - 3, qd = warp & 3, half = wi >> 2, tid = threadIdx.x - 96;
        int d_uses = 0;
        int64_t R = 0;             // passes exchanged
        const StepArgs &As = *A;
        const int RW = As.retire_width, strict = As.strict;
        // the call's pointers, read once (the head's stores could alias the argument block,
        // so the compiler would otherwise reload them from device memory every step)
        const uint8_t *const replay = As.replay;
        float *const pre_log = As.pre_log;
        uint8_t *const lat_log = As.lat_log;
        int64_t *const cycles_out = As.cycles_out;
        const uint32_t *const records = As.records;
        const bool prof = a.prof && blockIdx.x == 0 && tid == 0;
        uint64_t tp = prof ? (uint64_t)clock64() : 0;
        auto mark = [&](int k) {
            if (prof) {
                const uint64_t tn = (uint64_t)clock64();
                pacc[k] += tn - tp;
                tp = tn;
            }
        };
        auto signal = [&](int b) {   // this warp's share of a signal to the MMA warp (after its writes)
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(b));
        };
        // extent of this CTA's slots (longest queue + 1) and live count, to every CTA of the cluster
        auto send_ext = [&](int nb) {   // worker warp 0 only
            int mx = 0, al = 0;
            if (lane < SPC && s_al[lane]) { mx = s_ql[lane] + s_ml[lane] + 1; al = 1; }   // whole context
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                al += __shfl_xor_sync(0xffffffffu, al, o);
            }
            if (lane < CS) {   // one lane per destination CTA: the release arrives overlap
                cl_st_async_v2(cl_map(smem_u32(&ext_in[nb * CS + rank]), (uint32_t)lane), (uint32_t)mx, (uint32_t)al,
                               cl_map(bar(B_EXT + nb), (uint32_t)lane));
            }
            __syncwarp();
            if (lane == 0) xs[X_EXT_SENT] = xs[X_EXT_SENT] + 1;
        };
        if (wi == 0) send_ext(0);
        // feature rows of positions q0 .. q0 + P - 1 into the first layer's operand
        constexpr int NCH = F8 ? 4 : 8;   // 16-byte chunks of one 64-feature row
        auto chunks = [&](uint32_t rec, uint32_t cur, bool ctx, int32_t res, uint32_t e, uint32_t sl, uint4 (&o)[NCH]) {
            if constexpr (F8) row_chunks_fp8(rec, cur, ctx, res, e, sl, o);
            else row_chunks_bf16(rec, cur, ctx, res, e, sl, o);
        };
        auto build_rows = [&](int q0, int P) {
            // layer-0 A row (pair, slot), K = the pair's two rows: two 128-byte panels
            // (BF16) or the two halves of one (FP8)
            for (int f = tid; f < P * (1 << L) * SPC; f += kWk) {
                const int s = f % SPC, rr = f / SPC, r = q0 * (1 << L) + rr;
                const int m = (rr >> 1) * SPC + s;
                uint4 ch[NCH];
                const int ql = s_ql[s];
                // context row r: the processor queue newest first, then the write queue
                if (s_al[s] && r <= ql + s_ml[s]) {
                    const uint32_t cur = recb[s * 4 + (s_p[s] & 3)];
                    if (r == 0) {
                        chunks(cur, cur, false, 0, 0u, 0u, ch);
                    } else {
                        uint64_t ent;
                        if (r <= ql) {
                            int idx = s_qs[s] + ql - r;
                            if (idx >= cap) idx -= cap;
                            ent = qring[s * cap + idx];
                        } else {
                            int idx = s_ms[s] + s_ml[s] - (r - ql);
                            if (idx >= cap) idx -= cap;
                            ent = mring[s * cap + idx];
                        }
                        chunks(entry_rec(ent), cur, true, entry_res(ent, s_tick[s]), entry_e(ent), entry_s(ent), ch);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < NCH; j++) ch[j] = make_uint4(0, 0, 0, 0);
                }
                const int c0 = F8 ? 4 * (rr & 1) : 0;   // first chunk of this row in its operand row
                uint8_t *dst = sm + y.act + (uint32_t)(F8 ? 0 : (rr & 1)) * pstride_of(0, P) + (uint32_t)m * 128u;
#pragma unroll
                for (int j = 0; j < NCH; j++) *reinterpret_cast<uint4 *>(dst + (((c0 + j) ^ (m & 7)) << 4)) = ch[j];
            }
        };
        // Epilogue of layer l, channel half h, for this warp's TMEM lanes (quadrant qd) and its
        // quarter of the channels: bias, ReLU, rounding (FP8: dequantise and requantise), written
        // as the next layer's operand (rows 2j, 2j+1 of a slot side by side along K) or, after
        // the last conv layer, as this CTA's rows of the FC1 operand.
        auto epilogue = [&](auto CWc, int l, int P, int h) {
            constexpr int CW = decltype(CWc)::value;   // channels a warp converts (C / 4)
            const bool last = l == L - 1;
            const int T = tiles_of(l, P), Rl = rows_of(l, P);
            const int cb = h * (C / 2) + half * CW;   // this warp's first channel
            for (int tt = 0; tt < T; tt++) {
                const int m = tt * 128 + qd * 32 + lane;   // this lane's row of the tile
                if (tt * 128 + qd * 32 >= Rl) continue;    // warp-uniform: rows past the pass
                const bool valid = m < Rl;
                const int p = m / SPC, s = m % SPC;
                int row;
                uint32_t base, pstride;
                if (!last) {   // next layer's row (pair p >> 1, slot s), K half p & 1
                    row = (p >> 1) * SPC + s;
                    base = y.act;
                    pstride = pstride_of(l + 1, P);
                } else {       // FC1 operand: row = cluster slot, K = position in pass x C + channel
                    row = (int)rank * SPC + s;
                    base = y.fc1a;
                    pstride = 16384u;
                }
                const int kb = (last ? p * C : (p & 1) * C) + cb;
                uint32_t r[CW];
                const uint32_t ta = tmem_base + ((uint32_t)(qd * 32) << 16) + dcol(l) + (uint32_t)(tt * C + cb);
                if constexpr (CW == 32) tmem_ld32(ta, r);
                else tmem_ld16(ta, r);
                if constexpr (F8) {
                    // dequantise (weight scale), bias, ReLU and requantise to the next layer's
                    // input scale in one FMA (the scale folded into the weight scale and the
                    // bias at the start), e4m3 with saturation: 16 channels a chunk
                    const int cc = l * C + cb;
                    const float4 *cbv = reinterpret_cast<const float4 *>(s_cb + cc);
                    const float4 *cw = reinterpret_cast<const float4 *>(s_ws + cc);
                    uint32_t w[CW / 4];
#pragma unroll
                    for (int j = 0; j < CW / 4; j++) {
                        const float4 b = cbv[j], sw = cw[j];
                        const float v0 = fmaxf(__uint_as_float(r[4 * j]) * sw.x + b.x, 0.f);
                        const float v1 = fmaxf(__uint_as_float(r[4 * j + 1]) * sw.y + b.y, 0.f);
                        const float v2 = fmaxf(__uint_as_float(r[4 * j + 2]) * sw.z + b.z, 0.f);
                        const float v3 = fmaxf(__uint_as_float(r[4 * j + 3]) * sw.w + b.w, 0.f);
                        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v0, v1), __NV_SATFINITE, __NV_E4M3);
                        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v2, v3), __NV_SATFINITE, __NV_E4M3);
                        w[j] = (lo & 0xffffu) | (hi << 16);
                    }
#pragma unroll
                    for (int j = 0; j < CW / 16; j++) {
                        const int k = kb + 16 * j;
                        // FC1 operand with 128 channels: half panels of 64-byte rows (64-byte swizzle)
                        const uint32_t off = last && hfc
                                                 ? base + (uint32_t)(k >> 6) * 8192u + (uint32_t)row * 64u +
                                                       ((uint32_t)(((k >> 4) & 3) ^ ((row >> 1) & 3)) << 4)
                                                 : base + (uint32_t)(k >> 7) * pstride + (uint32_t)row * 128u +
                                                       ((uint32_t)(((k >> 4) & 7) ^ (row & 7)) << 4);
                        if (valid)
                            *reinterpret_cast<uint4 *>(sm + off) = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
                    }
                } else {
                    // bias four channels to a load; ReLU on the rounded pairs (rounding to
                    // nearest keeps the sign, so this equals rounding the ReLU output)
                    const float4 *cbv = reinterpret_cast<const float4 *>(s_cb + l * C + cb);
                    const __nv_bfloat162 zero2 = __floats2bfloat162_rn(0.f, 0.f);
                    uint32_t w[CW / 2];
#pragma unroll
                    for (int j = 0; j < CW / 4; j++) {
                        const float4 b = cbv[j];
                        __nv_bfloat162 p0 = __floats2bfloat162_rn(__uint_as_float(r[4 * j]) + b.x,
                                                                  __uint_as_float(r[4 * j + 1]) + b.y);
                        __nv_bfloat162 p1 = __floats2bfloat162_rn(__uint_as_float(r[4 * j + 2]) + b.z,
                                                                  __uint_as_float(r[4 * j + 3]) + b.w);
                        p0 = __hmax2(p0, zero2);
                        p1 = __hmax2(p1, zero2);
                        w[2 * j] = *reinterpret_cast<uint32_t *>(&p0);
                        w[2 * j + 1] = *reinterpret_cast<uint32_t *>(&p1);
                    }
#pragma unroll
                    for (int j = 0; j < CW / 8; j++) {
                        const int k = kb + 8 * j;
                        const uint32_t off = base + (uint32_t)(k >> 6) * pstride + (uint32_t)row * 128u +
                                             ((uint32_t)(((k >> 3) & 7) ^ (row & 7)) << 4);
                        if (valid)
                            *reinterpret_cast<uint4 *>(sm + off) = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
                    }
                }
            }
        };
        auto epi = [&](int l, int P, int h) {
            if (C == 128) epilogue(std::integral_constant<int, 32>{}, l, P, h);
            else epilogue(std::integral_constant<int, 16>{}, l, P, h);
        };
        // Epilogue of a swapped layer (TMEM lanes = output channels, columns = the pass's
        // rows): this warp takes 16 channels (half of its quadrant's lanes) of every row, 16
        // rows at a time: bias, ReLU and BF16 pairs in the 8x8 fragment layout the 16x256b
        // load delivers, stored transposed by stmatrix, i.e. as 16-byte runs of 8 channels of
        // one operand row (the same bytes the row-major epilogue writes).
        auto epi_swapped = [&](int l, int P) {
            const bool last = l == L - 1;
            const int Rl = rows_of(l, P);
            const int cob = qd * 32 + half * 16, g = lane >> 2;
            const float b0 = s_cb[l * C + cob + g], b1 = s_cb[l * C + cob + 8 + g];
            const uint32_t ta = tmem_base + ((uint32_t)cob << 16) + dcol(l);
            const int mi = lane >> 3, mj = lane & 7;              // the matrix and row this thread addresses
            const int cbi = cob + ((mi & 1) ? 8 : 0), rbo = (mi & 2) ? 8 : 0;
            const __nv_bfloat162 zero2 = __floats2bfloat162_rn(0.f, 0.f);
            auto pk = [&](uint32_t x, uint32_t y, float b) {
                __nv_bfloat162 v = __floats2bfloat162_rn(__uint_as_float(x) + b, __uint_as_float(y) + b);
                v = __hmax2(v, zero2);
                return *reinterpret_cast<uint32_t *>(&v);
            };
            for (int r0 = 0; r0 < Rl; r0 += 16) {
                uint32_t v[8];
                tmem_ld16x256b_x2(ta + (uint32_t)r0, v);
                const uint32_t f[4] = {pk(v[0], v[1], b0), pk(v[2], v[3], b1), pk(v[4], v[5], b0), pk(v[6], v[7], b1)};
                const int m = r0 + rbo + mj, p = m / SPC, s = m % SPC;
                int row, k;
                uint32_t base, pstride;
                if (!last) {   // next layer's row (pair p >> 1, slot s), K half p & 1
                    row = (p >> 1) * SPC + s;
                    k = (p & 1) * C + cbi;
                    base = y.act;
                    pstride = pstride_of(l + 1, P);
                } else {       // FC1 operand: row = cluster slot, K = position in pass x C + channel
                    row = (int)rank * SPC + s;
                    k = p * C + cbi;
                    base = y.fc1a;
                    pstride = 16384u;
                }
                const uint32_t off = base + (uint32_t)(k >> 6) * pstride + (uint32_t)row * 128u +
                                     ((uint32_t)(((k >> 3) & 7) ^ (row & 7)) << 4);
                stmatrix_x4_trans(smem_u32(sm + off), f);
            }
        };
        // this CTA's rows of the pass's FC1 panels of channel half h (all panels when a panel
        // spans both halves: h = 1 only) to every peer: lane j of worker warp 0 (whose TMEM
        // lanes hold no rows of a last layer with at most 96 rows) sends to peer rank + j, one
        // bulk copy per unit, counted on the peer's B_FULL + unit; a peer overwrites its copy
        // only after B_EMPTY, i.e. after every CTA's FC1 of this pass, which waited for all of
        // its copies
        auto send_rows = [&](int P, int h) {
            if (wi != 0 || lane < 1 || lane >= CS) return;
            const uint32_t peer = (rank + (uint32_t)lane) % CS;
            const int np = xunits(P);
            for (int i = 0; i < np; i++) {
                // units half a row wide (BF16 panels, FP8 half panels): the even ones are
                // complete after the first half
                if ((kSplit && EPP < C) || hfc ? (i & 1) != h : h == 0) continue;
                const uint32_t src = fc0 + (uint32_t)i * xstride + rank * xbytes;
                cl_bulk_copy(cl_map(src, peer), src, xbytes, cl_map(bar(B_FULL + i), peer));
            }
            if (h == 1) {
                xs[X_ROWS_SENT + lane] = (int)R + 1;   // what this lane sent its peer
                xs[X_ROWS_NP + lane] = np;
            }
        };
        // The first pass always covers P0 positions: its rows need no cluster-wide extent, so
        // they are built (and the first layer's MMAs issued) while the extents are exchanged
        // (positions of the pass past the extent are padding rows, computed rather than taken
        // from S[e]: the same result).
        const int P0 = min(PM, a.rows_n);
        uint32_t ph_ctl = 0;
        bool stop = false;
        for (int64_t t = 0; t < a.n_steps && !stop; t++) {
            workers_sync();   // the previous step's head (worker warp 0) is visible
            build_rows(0, P0);
            signal(B_ROWS);   // the MMA warp starts the first layer; the extent is read after it
            mark(0);
            int eL = P0;      // the first pass's positions, whatever the extent
            for (int q0 = 0; q0 < eL && !stop; q0 += PM) {
                const int P = min(PM, eL - q0);   // P0 for the first pass
                if (q0 > 0) {
                    build_rows(q0, P);
                    signal(B_ROWS);
                }
                mark(1);
                for (int l = 0; l < L; l++) {
                    const bool last = l == L - 1;
                    bool ok = note(sleep_wait(bar(B_D), (uint32_t)d_uses & 1u, lim, abort_f, a.status, false), 5, t, R);
                    d_uses++;
                    if (last && R >= 1 && ok) {   // every CTA has consumed the previous pass's exchanged rows
                        const uint64_t tb = prof ? (uint64_t)clock64() : 0;
                        ok = note(cl_wait(b_empty(R - 1), (uint32_t)(((R - 1) >> 1) & 1), lim, abort_f, a.status),
                                  6, t, R);
                        if (prof) pacc[13] += (uint64_t)clock64() - tb;
                    }
                    ok = __all_sync(0xffffffffu, ok);
                    tc_fence_after();
                    mark(2 + 2 * l);
                    if (swapped(l, P)) {
                        // both channel halves at once (each warp converts its own channels)
                        if (ok) epi_swapped(l, P);
                        tc_fence_before();
                        signal(B_HA);
                        signal(B_HB);
                        if (last) {
                            workers_sync();
                            if (ok) send_rows(P, 0);
                        }
                    } else {
                        // the first channel half, handed to the MMA warp (and its complete FC1
                        // panels to the peers) while the second is converted
                        if (ok) epi(l, P, 0);
                        tc_fence_before();
                        signal(B_HA);
                        if (last) {
                            workers_sync();
                            if (ok && ((kSplit && EPP < C) || hfc)) send_rows(P, 0);
                        }
                        if (ok) epi(l, P, 1);
                        tc_fence_before();
                        signal(B_HB);
                    }
                    if (q0 == 0 && l == 0) {
                        // the step's extent, published by the producer: positions, or the
                        // cluster is done (then the MMA warp stops before the second layer)
                        const bool w = note(sleep_wait(bar(B_CTL), ph_ctl, lim, abort_f, a.status, false), 14, t, R);
                        ph_ctl ^= 1u;
                        const volatile int *c = ctl + 2 * (int)(t & 1);
                        stop = workers_any(!w || c[1] != 0);   // the same decision in every worker
                        if (stop) break;
                        eL = c[0];
                        if (prof) { pacc[14] += 1; pacc[15] += (unsigned long long)eL; }
                        if (tid == 0 && rank == 0 && 2 * t >= a.n_steps) {   // extent in the launch's second half
                            atomicAdd(&a.pos_sum[0], (unsigned long long)eL);
                            atomicAdd(&a.pos_sum[1], 1ull);
                        }
                        if (tid >= 128 && tid < 128 + HN) {   // S[e] of this CTA's neurons, for the FC1 epilogue
                            cp_async4(smem_u32(&s_Se[tid - 128]), a.fc1_const + (size_t)eL * a.H + (int)rank * HN + (tid - 128));
                            cp_commit();
                        }
                    }
                    if (last) {
                        if (tid >= 128 && tid < 128 + HN) {   // S[e] landed; FC1's bias added once a step
                            cp_wait<0>();
                            if (q0 == 0) s_Se[tid - 128] += s_fb[tid - 128];
                        }
                        workers_sync();   // this CTA's rows of the pass are all in its own buffer
                        if (ok) send_rows(P, 1);
                        __syncwarp();
                        R++;
                    }
                    mark(3 + 2 * l);
                }
            }
            if (stop) break;
            // FC1 epilogue: ReLU(FC1 + bias + S[e]) folded into FC2 partials per slot
            {
                bool ok = note(sleep_wait(bar(B_DFC), (uint32_t)(t & 1), lim, abort_f, a.status, false), 8, t, R);
                ok = __all_sync(0xffffffffu, ok);
                tc_fence_after();
                mark(8);
                float pf = 0.f, pe = 0.f, ps = 0.f;
                constexpr int NH = NO <= 3 ? 1 : 24;
                float ph[NH];
#pragma unroll
                for (int o = 0; o < NH; o++) ph[o] = 0.f;
                if (ok) {
                    const int cols = HN / 2, j0 = half * cols;
                    if constexpr (NO <= 3) {
                        uint32_t r32[2][32];
                        tmem_ld_cols(tmem_base + ((uint32_t)(qd * 32) << 16) + 384u + (uint32_t)j0, cols, r32);
#pragma unroll
                        for (int bi = 0; bi < 2; bi++) {
                            if (bi >= cols / 32) break;
                            // bias + S[e] and FC2 rows four neurons to a load
                            const int jb = j0 + bi * 32;
                            const float4 *se4 = reinterpret_cast<const float4 *>(s_Se + jb);
                            const float4 *wf4 = reinterpret_cast<const float4 *>(s_w2f + jb);
                            const float4 *we4 = reinterpret_cast<const float4 *>(s_w2e + jb);
                            const float4 *ws4 = reinterpret_cast<const float4 *>(s_w2f + 2 * HN + jb);   // SQ only
                            const float4 *fw4 = reinterpret_cast<const float4 *>(s_fws + jb);            // FP8 only
#pragma unroll
                            for (int q = 0; q < 8; q++) {
                                const float4 se = se4[q], wf = wf4[q], we = we4[q];
                                float4 wsv = make_float4(0.f, 0.f, 0.f, 0.f), fsc = make_float4(1.f, 1.f, 1.f, 1.f);
                                if constexpr (SQ) wsv = ws4[q];
                                if constexpr (F8) fsc = fw4[q];
                                const float bb[4] = {se.x, se.y, se.z, se.w};
                                const float wfa[4] = {wf.x, wf.y, wf.z, wf.w}, wea[4] = {we.x, we.y, we.z, we.w};
                                const float wsa[4] = {wsv.x, wsv.y, wsv.z, wsv.w}, fsa[4] = {fsc.x, fsc.y, fsc.z, fsc.w};
#pragma unroll
                                for (int u = 0; u < 4; u++) {
                                    const float acc = __uint_as_float(r32[bi][4 * q + u]);
                                    const float v = fmaxf((F8 ? acc * fsa[u] : acc) + bb[u], 0.f);
                                    pf = fmaf(v, wfa[u], pf);
                                    pe = fmaf(v, wea[u], pe);
                                    if constexpr (SQ) ps = fmaf(v, wsa[u], ps);
                                }
                            }
                        }
                    } else {
                        // 22 outputs per neuron: 16 TMEM columns at a time keeps the
                        // accumulators and one chunk in registers (no spills)
#pragma unroll 1
                        for (int bi = 0; bi < cols / 16; bi++) {
                            uint32_t r32[16];
                            tmem_ld16(tmem_base + ((uint32_t)(qd * 32) << 16) + 384u + (uint32_t)(j0 + bi * 16), r32);
#pragma unroll
                            for (int jj = 0; jj < 16; jj++) {
                                const int j = j0 + bi * 16 + jj;
                                const float acc = __uint_as_float(r32[jj]) * (F8 ? s_fws[j] : 1.f);
                                const float v = fmaxf(acc + s_Se[j], 0.f);
                                const float4 *wv = reinterpret_cast<const float4 *>(s_w2 + j * 24);
#pragma unroll
                                for (int q4 = 0; q4 < 6; q4++) {
                                    const float4 w = wv[q4];
                                    ph[4 * q4] = fmaf(v, w.x, ph[4 * q4]);
                                    ph[4 * q4 + 1] = fmaf(v, w.y, ph[4 * q4 + 1]);
                                    if (4 * q4 + 2 < NO) ph[4 * q4 + 2] = fmaf(v, w.z, ph[4 * q4 + 2]);
                                    if (4 * q4 + 3 < NO) ph[4 * q4 + 3] = fmaf(v, w.w, ph[4 * q4 + 3]);
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                // cluster slot g = qd * 32 + lane belongs to CTA g / SPC, where it is slot g % SPC
                const uint64_t te0 = prof ? (uint64_t)clock64() : 0;
                if (prof) pacc[30] += te0 - tp;   // FC1 epilogue arithmetic (thread 0)
                const int g = qd * 32 + lane, owner = g / SPC;
                const uint32_t dst =
                    cl_map(smem_u32(&part[(((int)rank * 2 + half) * SPC + g % SPC) * PF]), (uint32_t)owner);
                const uint32_t pb = cl_map(bar(B_PART), (uint32_t)owner);
                if constexpr (NO == 2) {
                    cl_st_async_v2(dst, __float_as_uint(pf), __float_as_uint(pe), pb);
                } else if constexpr (SQ) {
                    cl_st_async_v4(dst, make_uint4(__float_as_uint(pf), __float_as_uint(pe), __float_as_uint(ps), 0u), pb);
                } else {
#pragma unroll
                    for (int q4 = 0; q4 < 6; q4++)
                        cl_st_async_v4(dst + 16u * q4,
                                       make_uint4(__float_as_uint(ph[4 * q4]), __float_as_uint(ph[4 * q4 + 1]),
                                                  __float_as_uint(ph[4 * q4 + 2]), __float_as_uint(ph[4 * q4 + 3])),
                                       pb);
                }
                if (tid == 0) xs[X_PART_SENT] = xs[X_PART_SENT] + 1;   // every worker sent its share
                if (prof) pacc[31] += (uint64_t)clock64() - te0;   // partial sums to their owners
                mark(9);
            }
            // head, clock and queue update, drain: one thread per slot (warp 2)
            if (wi == 0) {
                bool ok = note(sleep_wait(bar(B_PART), (uint32_t)(t & 1), lim, abort_f, a.status, true), 9, t, R);
                if (ok && lane == 0) {
                    mbar_expect_tx(bar(B_PART), kPartBytes);   // the next step's phase
                    xs[X_PART_CONS] = xs[X_PART_CONS] + 1;
                }
                ok = __all_sync(0xffffffffu, ok);
                mark(10);
                const int s = lane;
                if (ok && s < SPC && s_al[s]) {
                    const int64_t o = s_o[s];
                    const int n = s_n[s];
                    int p = s_p[s];
                    float z[NO];
                    if constexpr (NO == 2) {
                        float zf = s_b2[0], ze = s_b2[1];
#pragma unroll
                        for (int i = 0; i < 2 * CS; i++) {
                            const float2 v = reinterpret_cast<const float2 *>(part)[i * SPC + s];
                            zf += v.x;
                            ze += v.y;
                        }
                        z[0] = zf;
                        z[1] = ze;
                    } else if constexpr (SQ) {
#pragma unroll
                        for (int o2 = 0; o2 < NO; o2++) z[o2] = s_b2[o2];
#pragma unroll
                        for (int i = 0; i < 2 * CS; i++) {
                            const float4 v = reinterpret_cast<const float4 *>(part)[i * SPC + s];
                            z[0] += v.x;
                            z[1] += v.y;
                            z[min(2, NO - 1)] += v.z;
                        }
                    } else {
#pragma unroll
                        for (int o2 = 0; o2 < NO; o2++) z[o2] = s_b2[o2];
#pragma unroll
                        for (int i = 0; i < 2 * CS; i++) {
                            const float *pv = part + (i * SPC + s) * PF;
#pragma unroll
                            for (int q4 = 0; q4 < 6; q4++) {
                                const float4 v = *reinterpret_cast<const float4 *>(pv + 4 * q4);
                                z[4 * q4] += v.x;
                                z[4 * q4 + 1] += v.y;
                                if (4 * q4 + 2 < NO) z[min(4 * q4 + 2, NO - 1)] += v.z;
                                if (4 * q4 + 3 < NO) z[min(4 * q4 + 3, NO - 1)] += v.w;
                            }
                        }
                    }
                    float yf, ye, ys = 0.f;
                    uint32_t F = head_latency<NO, 0>(z, yf), E = head_latency<NO, 1>(z, ye), Sl = 0;
                    if constexpr (SQ) Sl = head_latency<NO, 2>(z, ys);
                    const int64_t gi = o + p;
                    if (replay) {
                        F = replay[NL * gi];
                        E = replay[NL * gi + 1];
                        if constexpr (SQ) Sl = replay[NL * gi + 2];
                    }
                    if (pre_log) {
                        pre_log[NL * gi] = yf;
                        pre_log[NL * gi + 1] = ye;
                        if constexpr (SQ) pre_log[NL * gi + 2] = ys;
                    }
                    if (lat_log) {
                        lat_log[NL * gi] = (uint8_t)F;
                        lat_log[NL * gi + 1] = (uint8_t)E;
                        if constexpr (SQ) lat_log[NL * gi + 2] = (uint8_t)Sl;
                    }
                    uint64_t *qr = qring + s * cap;
                    uint64_t *mr = mring + s * cap;   // SQ only
                    int qs = s_qs[s], ql = s_ql[s], ev = 0;
                    int ms = SQ ? s_ms[s] : 0, ml = SQ ? s_ml[s] : 0;
                    int32_t tick = s_tick[s] + (int32_t)F;
                    // in-order retire from the oldest, at most lim_n entries; with the store
                    // latency the retired stores move to the write queue's tail, and the write
                    // queue then retires in order, with no limit, every store whose residence
                    // has reached its S
                    auto retire = [&](int lim_n) {
                        // four entries a round: their loads are independent and overlap, the
                        // tests then run in order (a ring load costs ~30 cycles, a round of
                        // one entry ~50)
                        int k = 0;
                        bool blocked = false;
                        while (k < lim_n && !blocked) {
                            uint64_t v[4];
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                int idx = qs + k + u;   // below 2 cap for the entries tested
                                if (idx >= cap) idx -= cap;
                                v[u] = qr[min(idx, cap - 1)];
                            }
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                if (blocked || k >= lim_n) break;
                                const int32_t res = entry_res(v[u], tick), e = (int32_t)entry_e(v[u]);
                                if (strict ? res <= e : res < e) {
                                    blocked = true;
                                    break;
                                }
                                if constexpr (SQ) {
                                    if (rec_is_store(entry_rec(v[u]))) {
                                        int mi = ms + ml;
                                        if (mi >= cap) mi -= cap;
                                        mr[mi] = v[u];
                                        ml++;
                                    }
                                }
                                k++;
                            }
                        }
                        qs += k;
                        if (qs >= cap) qs -= cap;
                        ql -= k;
                        if constexpr (SQ) {
                            int km = 0;
                            while (km < ml) {
                                int idx = ms + km;
                                if (idx >= cap) idx -= cap;
                                const uint64_t v = mr[idx];
                                const int32_t res = entry_res(v, tick), sl = (int32_t)entry_s(v);
                                if (strict ? res <= sl : res < sl) break;
                                km++;
                            }
                            ms += km;
                            if (ms >= cap) ms -= cap;
                            ml -= km;
                        }
                    };
                    retire(min(ql, RW * (int)F));
                    if (ql + ml == cap) {   // full: drop the oldest instruction (the write queue's head first)
                        if (SQ && ml > 0) {
                            ms = (ms + 1 == cap) ? 0 : ms + 1;
                            ml--;
                        } else {
                            qs = (qs + 1 == cap) ? 0 : qs + 1;
                            ql--;
                        }
                        ev = 1;
                    }
                    {
                        int idx = qs + ql;
                        if (idx >= cap) idx -= cap;
                        qr[idx] = pack_entry(recb[s * 4 + (p & 3)], E, SQ ? Sl : 0u, (uint32_t)tick);
                    }
                    ql++;
                    p++;
                    if (p == n) {   // drain: Delta of Eq. 1
                        while (ql + ml > 0) {
                            tick += 1;
                            retire(min(ql, RW));
                        }
                        cycles_out[s_b[s]] = tick;
                    }
                    s_tick[s] = tick;
                    s_p[s] = p;
                    s_qs[s] = qs;
                    s_ql[s] = ql;
                    if constexpr (SQ) {
                        s_ms[s] = ms;
                        s_ml[s] = ml;
                    }
                    s_ev[s] += ev;
                    s_al[s] = p < n ? 1 : 0;
                    if (p + 1 < n)   // record of the position two steps ahead
                        cp_async4(smem_u32(&recb[s * 4 + ((p + 1) & 3)]), records + o + p + 1);
                }
                cp_commit();      // one group per step, empty or not
                cp_wait<1>();     // the record fetched one step ago has landed
                mark(11);
                __syncwarp();
                send_ext((int)((t + 1) & 1));
                mark(12);
            }
        }
        // state back to device memory (resumable), outstanding record copies drained; the
        // barrier orders the last step's head (warp 2) before the other warps read its state
        cp_wait<0>();
        workers_sync();
        for (int j = 0; j < SPC / 8; j++) {
            const int s = wi + 8 * j, b = s_b[s];
            if (b < 0) continue;
            for (int i = lane; i < cap; i += 32) A->ring[(size_t)b * cap + i] = qring[s * cap + i];
            if constexpr (SQ)
                for (int i = lane; i < cap; i += 32) A->mring[(size_t)b * cap + i] = mring[s * cap + i];
            if (lane == 0) {
                A->tick[b] = s_tick[s];
                A->pos[b] = s_p[s];
                A->qstart[b] = s_qs[s];
                A->qlen[b] = s_ql[s];
                if constexpr (SQ) {
                    A->mstart[b] = s_ms[s];
                    A->mlen[b] = s_ml[s];
                }
                A->evict[b] = s_ev[s];
            }
        }
    } else if (lane == 0) {
        // ---------------------------------------------------------------- warp 1: FC1 done
        // Once this CTA's FC1 MMAs of a pass have completed, its copy of the pass's rows
        // may be overwritten: one arrive on every CTA's B_EMPTY + (pass & 1).
        int rh = 0;
        uint64_t t0 = gtimer();
        while (true) {
            if (try_sleep(bar(B_F1D), (uint32_t)(rh & 1), 20000u, false)) {
                for (int r = 0; r < CS; r++) cl_arrive_remote(cl_map(b_empty(rh), (uint32_t)r));
                rh++;
                t0 = gtimer();
                continue;
            }
            if (xs[X_DONE] && rh >= xs[X_F1C]) break;
            if ((int64_t)(gtimer() - t0) > lim) {
                *abort_f = 1;
                atomicExch(a.status, kStatusTimeout);
                note(false, 10, -1, rh);
                break;
            }
        }
    }
    __syncthreads();
    if (a.prof && blockIdx.x == 0 && threadIdx.x < 32) a.prof[threadIdx.x] = pacc[threadIdx.x];
    if (warp == 0 && lane == 0) {   // weight panels issued but never consumed (early exit) land first
        for (int it = cnt[1]; it < cnt[0]; it++) drain_wait(bar(it % S), (uint32_t)(it / S) & 1u, drain_ns);
    }
    __syncthreads();
    // Leaving.  Every peer learns what this CTA sent it: extents and partial-sum
    // steps, and the passes (and their panel count) of row copies.
    if (threadIdx.x < CS) {
        const int d = (int)threadIdx.x, wd = (d - (int)rank + CS) % CS;   // the lane that sends to d
        const uint4 v = make_uint4((uint32_t)xs[X_EXT_SENT], (uint32_t)xs[X_PART_SENT],
                                   wd ? (uint32_t)xs[X_ROWS_SENT + wd] : 0u, wd ? (uint32_t)xs[X_ROWS_NP + wd] : 0u);
        cl_st_v4(cl_map(smem_u32(&inbox[rank]), (uint32_t)d), v);
    }
    cluster_sync_all();   // the counts are in, and no CTA starts another write into a peer
    if (threadIdx.x == 0) {
        // Wait, on the barriers they complete on, until every write sent to this CTA
        // has landed.  A phase that was armed for bytes no peer sent gets them
        // completed here; one that was not armed is armed for what was sent.
        // Extents: phases of the steps after the last one consumed (armed two ahead);
        // partial sums: the step after the last one consumed; rows: the pass after the
        // last one whose FC1 read them all (peers send a pass only after every CTA's
        // FC1 of the previous one), every panel whose phase the FC1 MMAs did not wait for.
        const int tc = xs[X_EXT_CONS];
        for (int st = tc; st < tc + 2; st++) {
            uint32_t got = 0;
            for (int q = 0; q < CS; q++)
                if ((int)inbox[q].x > st) got += 8u;
            const uint32_t b = bar(B_EXT + (st & 1));
            if (got < kExtBytes) mbar_complete_tx(b, kExtBytes - got);
            drain_wait(b, (uint32_t)(st >> 1) & 1u, drain_ns);
        }
        const int pc = xs[X_PART_CONS];
        uint32_t got = 0;
        for (int q = 0; q < CS; q++)
            if ((int)inbox[q].y > pc) got += kPartBytes / CS;
        if (got < kPartBytes) mbar_complete_tx(bar(B_PART), kPartBytes - got);
        drain_wait(bar(B_PART), (uint32_t)pc & 1u, drain_ns);
        const int rc = xs[X_ROWS_DONE];
        int senders = 0, np = 0;
        for (int q = 0; q < CS; q++)
            if (q != (int)rank && (int)inbox[q].z > rc) {
                senders++;
                np = (int)inbox[q].w;
            }
        const bool armed = xs[X_ARMED_R] > rc;
        if (armed) np = xs[X_ARMED_NP];
        const uint32_t fph_now = (uint32_t)xs[X_FPH], waited = armed ? (uint32_t)xs[X_FC1_WAITED] : 0u;
        for (int i = 0; i < np; i++) {
            if ((waited >> i) & 1u) continue;   // its phase completed in the FC1 MMAs
            const uint32_t b = bar(B_FULL + i);
            if (armed) {
                const uint32_t missing = (uint32_t)(CS - 1 - senders) * xbytes;
                if (missing) mbar_complete_tx(b, missing);
            } else if (senders > 0) {
                mbar_expect_tx(b, (uint32_t)senders * xbytes);
            } else {
                continue;
            }
            drain_wait(b, (fph_now >> i) & 1u, drain_ns);
        }
    }
    __syncthreads();
    cluster_sync_all();   // every copy into any CTA of the cluster has landed: none reads or writes here any more
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

// Cluster size: 8 CTAs (16 slots each) when FC1 still gives each at least 64
// neurons and the batch's clusters of 8 all fit on the GPU at once (every
// cluster keeps its sub-traces for the whole call, so clusters that wait for
// a free SM would run after the others); else 4 (32 slots each).
static int cluster_size(const simnet_config &k, int B) {
    if (k.fc_hidden / 8 < 64) return 4;
    const int n_clusters = (B + 127) / 128;
    return n_clusters * 8 <= num_sms() ? 8 : 4;
}

static int elem_bytes(const simnet_ctx *c) { return c->cfg.precision == SIMNET_FP8_E4M3 ? 1 : 2; }

// Shapes this kernel handles: BF16 or FP8 e4m3; 2 or 3 conv layers of 64 or 128
// channels; FC1 width 256 or 512; queue capacity below 256; the memory write
// queue only with the regression head.
bool cluster_eligible(const simnet_ctx *c, std::string &why) {
    const simnet_config &k = c->cfg;
    if (k.precision != SIMNET_BF16 && k.precision != SIMNET_FP8_E4M3) { why = "not BF16 or FP8"; return false; }
    if (c->store_queue && c->hybrid) { why = "memory write queue with the hybrid head"; return false; }
    if (c->residual) { why = "residual blocks"; return false; }
    if (k.n_conv < 2 || k.n_conv > 3) { why = "conv depth"; return false; }
    if (k.conv_channels != 64 && k.conv_channels != 128) { why = "conv width"; return false; }
    if (k.fc_hidden != 256 && k.fc_hidden != 512) { why = "FC1 width"; return false; }
    if (c->cap > 255 || c->rows_n < 1) { why = "window"; return false; }
    if ((c->rows_n * k.conv_channels * elem_bytes(c)) % 128 != 0) { why = "FC1 input not whole 128-byte panels"; return false; }
    const CLay y = c_layout(4, k.n_conv, k.conv_channels, k.fc_hidden, c->cap, 2, c->n_out, kPanelMax,
                            elem_bytes(c));   // the larger layout
    if (y.total + 1024 > 232448) { why = "shared memory"; return false; }
    return true;
}

// Largest stage count for a cluster size and stage size (0 if none fits).
static int cluster_stages_max(const simnet_ctx *c, int CS, int stage_bytes) {
    const simnet_config &k = c->cfg;
    int st = 8;
    while (st >= 2 && c_layout(CS, k.n_conv, k.conv_channels, k.fc_hidden, c->cap, st, c->n_out, stage_bytes,
                               elem_bytes(c)).total + 1024 > 232448)
        st--;
    return st >= 2 ? st : 0;
}

bool cluster_size_ok(const simnet_ctx *c, int CS, int B) {
    if (CS == 4) return true;
    return CS == 8 && c->cfg.fc_hidden / 8 >= 64 && (B + 127) / 128 * 8 <= num_sms();
}

int cluster_stage_limit(const simnet_ctx *c, int CS, int stage_bytes) { return cluster_stages_max(c, CS, stage_bytes); }

bool launch_cluster(simnet_ctx *c, int B, int64_t n_steps, cudaStream_t s, std::string &why) {
    if (!cluster_eligible(c, why)) return false;
    const simnet_config &k = c->cfg;
    const bool tuned = c->tuned_B == B;
    const int CS = tuned && c->tuned_cluster_size && cluster_size_ok(c, c->tuned_cluster_size, B)
                       ? c->tuned_cluster_size : cluster_size(k, B);
    CArgs a;
    memset(&a, 0, sizeof a);
    a.L = k.n_conv;
    a.C = k.conv_channels;
    a.H = k.fc_hidden;
    a.cap = c->cap;
    a.rows_n = c->rows_n;
    const int prec = k.precision, es = elem_bytes(c), epp = 128 / es;   // elements per 128-byte row
    const bool f8 = prec == SIMNET_FP8_E4M3;
    for (int l = 0; l < a.L; l++) {
        if (!encode_map_2d(a.tW[l], prec, c->Wl[l], (uint64_t)c->layer[l].K, (uint64_t)a.C, (uint32_t)epp,
                           (uint32_t)a.C, why))
            return false;
        a.cbias[l] = c->bias[l];
        a.cws[l] = f8 ? c->wscale[l] : nullptr;
        a.cos[l] = f8 ? c->oscale[l] : nullptr;
    }
    if (!encode_map_2d(a.tF, prec, c->Wl[a.L], (uint64_t)c->fc1_in, (uint64_t)a.H, (uint32_t)epp, (uint32_t)(a.H / CS),
                       why))
        return false;
    a.fws = f8 ? c->wscale[a.L] : nullptr;
    a.fbias = c->bias[a.L];
    a.w2 = c->w2;
    a.b2 = c->b2;
    a.fc1_const = c->fc1_const;
    a.A = c->d_args;
    a.status = c->status;
    a.prof = c->phase_on ? c->phase_ns : nullptr;
    a.tinfo = c->phase_ns + 48;
    a.pos_sum = c->phase_ns + 56;
    if (cudaMemsetAsync(a.tinfo, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess) { why = "memset"; return false; }
    a.n_steps = n_steps;
    a.spin_ns = c->cfg.spin_limit_ns;
    int stages = 8;
    const int no = c->n_out;
    auto fits = [&](int st, int sb) { return c_layout(CS, a.L, a.C, a.H, a.cap, st, no, sb, es).total + 1024 <= 232448; };
    a.stage_bytes = fits(3, 2 * kPanelMax) ? 2 * kPanelMax : kPanelMax;
    if (tuned && (c->tuned_cluster_stage_bytes == kPanelMax || c->tuned_cluster_stage_bytes == 2 * kPanelMax) &&
        fits(2, c->tuned_cluster_stage_bytes))
        a.stage_bytes = c->tuned_cluster_stage_bytes;   // the autotuner's pick
    while (stages > 2 && !fits(stages, a.stage_bytes)) stages--;
    if (tuned && c->tuned_cluster_stages >= 2 && c->tuned_cluster_stages < stages) stages = c->tuned_cluster_stages;
    a.stages = stages;
    const size_t smem = c_layout(CS, a.L, a.C, a.H, a.cap, stages, no, a.stage_bytes, es).total + 1024;
    void (*kern)(CArgs);
    if (f8)
        kern = no == kOutHybrid ? (CS == 8 ? cluster_kernel<8, kOutHybrid, true> : cluster_kernel<4, kOutHybrid, true>)
               : no == 3        ? (CS == 8 ? cluster_kernel<8, 3, true> : cluster_kernel<4, 3, true>)
                                : (CS == 8 ? cluster_kernel<8, 2, true> : cluster_kernel<4, 2, true>);
    else
        kern = no == kOutHybrid ? (CS == 8 ? cluster_kernel<8, kOutHybrid, false> : cluster_kernel<4, kOutHybrid, false>)
               : no == 3        ? (CS == 8 ? cluster_kernel<8, 3, false> : cluster_kernel<4, 3, false>)
                                : (CS == 8 ? cluster_kernel<8, 2, false> : cluster_kernel<4, 2, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return false; }
    const int n_clusters = (B + 127) / 128;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * CS);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return false; }
    return true;
}

}  // namespace simnet
