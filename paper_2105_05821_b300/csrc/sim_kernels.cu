// sim_kernels.cu -- per-step simulation kernels: context gather (Sec. 2.2), the
// latency head and the processor-queue / curTick update (Sec. 3.2), the drain
// of Eq. 1 (Sec. 3.1), active-set compaction for uneven sub-traces (Sec. 3.3).
#include "common.cuh"
#include "kernels.cuh"

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

// One thread per (slot, row, 16-byte chunk).  Row 0 = current instruction,
// row j = j-th newest queue entry, rows past the queue length are zero, and an
// inactive slot (sub-trace finished) gets all-zero rows.
template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(const StepArgs *__restrict__ A, T *__restrict__ X,
                                                     int n_slots) {
    constexpr int V = Vec<T>::N, CH = kNFP / V;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int W = A->window;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_slots * W * CH;
    if (gid >= total) return;
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
                for (int j = 0; j < V; j++) v[j] = feature(chunk * V + j, cur, cur, false, 0, 0);
            } else if (r <= A->qlen[b]) {
                const int cap = A->cap;
                int idx = A->qstart[b] + A->qlen[b] - r;
                if (idx >= cap) idx -= cap;
                const uint64_t ent = A->ring[(size_t)b * cap + idx];
                const int32_t res = A->tick[b] - (int32_t)entry_tick(ent);
                const uint32_t rec = entry_rec(ent), e = entry_e(ent);
#pragma unroll
                for (int j = 0; j < V; j++) v[j] = feature(chunk * V + j, rec, cur, true, res, e);
            }
        }
    }
    store16<T>(X + rowid * kNFP + chunk * V, v);
}

// Convert caller feature matrices [n][W][50] (float) into the device layout [n][W][64].
template <typename T>
__global__ void __launch_bounds__(256) pack_x_kernel(const float *__restrict__ x, T *__restrict__ X,
                                                     int64_t rows) {
    constexpr int V = Vec<T>::N, CH = kNFP / V;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= rows * CH) return;
    const int chunk = (int)(gid % CH);
    const int64_t row = gid / CH;
    float v[V];
#pragma unroll
    for (int j = 0; j < V; j++) {
        const int c = chunk * V + j;
        v[j] = c < kNF ? x[row * kNF + c] : 0.f;
    }
    store16<T>(X + row * kNFP + chunk * V, v);
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

// Length of the run of ready entries from the oldest, at most `lim`; in-order
// retire means the first not-ready entry stops it.  Whole warp participates.
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
            const int32_t res = tick - (int32_t)entry_tick(v);
            const int32_t e = (int32_t)entry_e(v);
            rd = strict ? (res > e) : (res >= e);
        }
        const unsigned m = __ballot_sync(0xffffffffu, rd);
        const int run = (m == 0xffffffffu) ? 32 : (__ffs(~m) - 1);
        k += run;
        if (run < 32) break;
    }
    return min(k, lim);
}

// One warp per active slot.  FC2 arrives as P partial dot products (one per
// FC1 column block) which are summed with the bias; softplus, clamp, round;
// then curTick += F, retire (budget RW*F), evict at capacity, append with
// residence 0; after the last instruction, drain one cycle at a time (budget
// RW) and write the sub-trace's cycle count.  Otherwise the warp writes the
// slot's feature rows for the next step (the gather, fused here).
template <typename T>
__global__ void __launch_bounds__(256) head_update_kernel(const StepArgs *__restrict__ A,
                                                          const float2 *__restrict__ part, int P,
                                                          int part_stride, const float *__restrict__ b2,
                                                          T *__restrict__ X) {
    __shared__ uint64_t s_ring[8][256];   // newest-first queue copy per warp (capacity <= 255)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int slot = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (slot >= *A->n_active) return;
    const int b = A->active[slot];
    const int64_t o = A->offsets[b], n = A->offsets[b + 1] - o;
    int p = A->pos[b];
    if (p >= n) return;
    float zf = 0.f, ze = 0.f;
    for (int i = lane; i < P; i += 32) {
        const float2 v = part[(size_t)i * part_stride + slot];
        zf += v.x;
        ze += v.y;
    }
    zf = warp_sum(zf) + b2[0];
    ze = warp_sum(ze) + b2[1];
    const float yf = softplus_f(zf), ye = softplus_f(ze);
    const int64_t gi = o + p;
    uint32_t F, E;
    if (A->replay) {
        F = A->replay[2 * gi];
        E = A->replay[2 * gi + 1];
    } else {
        F = to_cycles(yf);
        E = to_cycles(ye);
    }
    if (lane == 0) {
        if (A->pre_log) { A->pre_log[2 * gi] = yf; A->pre_log[2 * gi + 1] = ye; }
        if (A->lat_log) { A->lat_log[2 * gi] = (uint8_t)F; A->lat_log[2 * gi + 1] = (uint8_t)E; }
    }
    const int cap = A->cap, RW = A->retire_width, strict = A->strict;
    uint64_t *ring = A->ring + (size_t)b * cap;
    int qs = A->qstart[b], ql = A->qlen[b], ev = 0;
    int32_t tick = A->tick[b] + (int32_t)F;
    const int k = retire_run(ring, cap, qs, min(ql, RW * (int)F), tick, strict, lane);
    qs += k;
    if (qs >= cap) qs -= cap;
    ql -= k;
    if (ql == cap) {  // full: drop the oldest
        qs = (qs + 1 == cap) ? 0 : qs + 1;
        ql--;
        ev = 1;
    }
    if (lane == 0) {
        int idx = qs + ql;
        if (idx >= cap) idx -= cap;
        ring[idx] = pack_entry(A->records[gi], E, (uint32_t)tick);
    }
    ql++;
    p++;
    __syncwarp();
    if (p == n) {  // drain: Delta of Eq. 1
        while (ql > 0) {
            tick += 1;
            const int kk = retire_run(ring, cap, qs, min(ql, RW), tick, strict, lane);
            qs += kk;
            if (qs >= cap) qs -= cap;
            ql -= kk;
        }
        if (lane == 0) A->cycles_out[b] = tick;
    } else if (X) {
        // next step's input rows of this slot: row 0 = instruction p, row r = r-th newest entry.
        // The queue is copied newest-first into shared memory with independent loads first.
        uint64_t *sq = s_ring[threadIdx.x >> 5];
        for (int r = lane + 1; r <= ql; r += 32) {
            int idx = qs + ql - r;
            if (idx >= cap) idx -= cap;
            sq[r] = ring[idx];
        }
        __syncwarp();
        constexpr int V = Vec<T>::N, CH = kNFP / V, RPP = 32 / CH;
        const int W = A->window;
        const uint32_t cur = A->records[o + p];
        const int chunk = lane % CH;
        T *xs = X + (size_t)slot * W * kNFP;
        for (int r0 = 0; r0 < W; r0 += RPP) {
            const int r = r0 + lane / CH;
            float v[V];
#pragma unroll
            for (int j = 0; j < V; j++) v[j] = 0.f;
            if (r == 0) {
#pragma unroll
                for (int j = 0; j < V; j++) v[j] = feature(chunk * V + j, cur, cur, false, 0, 0);
            } else if (r <= ql) {
                const uint64_t ent = sq[r];
                const int32_t res = tick - (int32_t)entry_tick(ent);
                const uint32_t rec = entry_rec(ent), e = entry_e(ent);
#pragma unroll
                for (int j = 0; j < V; j++) v[j] = feature(chunk * V + j, rec, cur, true, res, e);
            }
            if (r < W) store16<T>(xs + (size_t)r * kNFP + chunk * V, v);
        }
    }
    if (lane == 0) {
        A->tick[b] = tick;
        A->pos[b] = p;
        A->qstart[b] = qs;
        A->qlen[b] = ql;
        A->evict[b] += ev;
    }
}

// FC2 from partial dot products: z = b2 + sum of P partials (pre-softplus), one warp per row.
__global__ void __launch_bounds__(256) head_part_z_kernel(const float2 *__restrict__ part, int P, int part_stride,
                                                          const float *__restrict__ b2, float *__restrict__ z,
                                                          int n) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float zf = 0.f, ze = 0.f;
    for (int i = lane; i < P; i += 32) {
        const float2 v = part[(size_t)i * part_stride + row];
        zf += v.x;
        ze += v.y;
    }
    zf = warp_sum(zf);
    ze = warp_sum(ze);
    if (lane == 0) {
        z[2 * row] = zf + b2[0];
        z[2 * row + 1] = ze + b2[1];
    }
}

// FC2 only (pre-softplus outputs) for the CNN-only entry point.
__global__ void __launch_bounds__(256) head_z_kernel(const float *__restrict__ h, const float *__restrict__ w2,
                                                     const float *__restrict__ b2, float *__restrict__ z,
                                                     int n, int H) {
    const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *hv = h + (size_t)row * H;
    float zf = 0.f, ze = 0.f;
    for (int j = lane; j < H; j += 32) {
        zf = fmaf(hv[j], w2[j], zf);
        ze = fmaf(hv[j], w2[H + j], ze);
    }
    zf = warp_sum(zf);
    ze = warp_sum(ze);
    if (lane == 0) {
        z[2 * row] = zf + b2[0];
        z[2 * row + 1] = ze + b2[1];
    }
}

// ------------------------------------------------------------------ set-up, compaction, totals
__global__ void init_state_kernel(const StepArgs *__restrict__ A) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) { *A->n_active = A->n_sub; *A->status = kStatusOk; }
    if (b >= A->n_sub) return;
    A->tick[b] = 0;
    A->pos[b] = 0;
    A->qstart[b] = 0;
    A->qlen[b] = 0;
    A->evict[b] = 0;
    A->active[b] = b;
    A->cycles_out[b] = 0;
}

// Stable in-place compaction of the active list: drop finished sub-traces so the
// batch stays dense.  One block.
__global__ void __launch_bounds__(1024) compact_kernel(const StepArgs *__restrict__ A) {
    __shared__ int wsum[32];
    __shared__ int base;
    asm volatile("griddepcontrol.wait;" ::: "memory");
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

__global__ void totals_kernel(const StepArgs *__restrict__ A, unsigned long long *__restrict__ out) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    unsigned long long cyc = 0, ev = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < A->n_sub; b += gridDim.x * blockDim.x) {
        cyc += (unsigned long long)A->cycles_out[b];
        ev += (unsigned long long)A->evict[b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cyc += __shfl_xor_sync(0xffffffffu, cyc, o);
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, cyc);
        atomicAdd(out + 1, ev);
    }
}

// Per-column maximum of non-negative values y [rows][C] into out[C] (float bits;
// monotone as unsigned for x >= 0).  Used by the FP8 calibration pass.
__global__ void channel_amax_kernel(const float *__restrict__ y, int64_t rows, int C, unsigned *__restrict__ out) {
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float m = 0.f;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) m = fmaxf(m, fabsf(y[r * C + c]));
    atomicMax(out + c, __float_as_uint(m));
}

// ------------------------------------------------------------------ launchers
void launch_channel_amax(const float *y, int64_t rows, int C, unsigned *out, cudaStream_t s) {
    dim3 g(128, (C + 127) / 128);
    channel_amax_kernel<<<g, 128, 0, s>>>(y, rows, C, out);
}

template <typename T>
void launch_gather(const StepArgs *A, T *X, int n_slots, int window, cudaStream_t s, bool pdl) {
    const int64_t total = (int64_t)n_slots * window * (kNFP / Vec<T>::N);
    launch_k(pdl, gather_kernel<T>, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, s, A, X, n_slots);
}
template void launch_gather<float>(const StepArgs *, float *, int, int, cudaStream_t, bool);
template void launch_gather<__nv_bfloat16>(const StepArgs *, __nv_bfloat16 *, int, int, cudaStream_t, bool);
template void launch_gather<__nv_fp8_e4m3>(const StepArgs *, __nv_fp8_e4m3 *, int, int, cudaStream_t, bool);

template <typename T>
void launch_pack_x(const float *x, T *X, int64_t rows, cudaStream_t s) {
    const int64_t total = rows * (kNFP / Vec<T>::N);
    if (total > 0) pack_x_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(x, X, rows);
}
template void launch_pack_x<float>(const float *, float *, int64_t, cudaStream_t);
template void launch_pack_x<__nv_bfloat16>(const float *, __nv_bfloat16 *, int64_t, cudaStream_t);
template void launch_pack_x<__nv_fp8_e4m3>(const float *, __nv_fp8_e4m3 *, int64_t, cudaStream_t);

template <typename T>
void launch_head_update(const StepArgs *A, const float2 *part, int P, int part_stride, const float *b2, T *X,
                        int n_slots, cudaStream_t s, bool pdl) {
    const int64_t threads = (int64_t)n_slots * 32;
    launch_k(pdl, head_update_kernel<T>, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, s, A, part, P,
             part_stride, b2, X);
}
template void launch_head_update<float>(const StepArgs *, const float2 *, int, int, const float *, float *, int,
                                        cudaStream_t, bool);
template void launch_head_update<__nv_bfloat16>(const StepArgs *, const float2 *, int, int, const float *,
                                                __nv_bfloat16 *, int, cudaStream_t, bool);
template void launch_head_update<__nv_fp8_e4m3>(const StepArgs *, const float2 *, int, int, const float *,
                                                __nv_fp8_e4m3 *, int, cudaStream_t, bool);

void launch_head_z(const float *h, const float *w2, const float *b2, float *z, int n, int H, cudaStream_t s) {
    const int64_t threads = (int64_t)n * 32;
    if (n > 0) head_z_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(h, w2, b2, z, n, H);
}

void launch_head_part_z(const float2 *part, int P, int part_stride, const float *b2, float *z, int n,
                        cudaStream_t s) {
    const int64_t threads = (int64_t)n * 32;
    if (n > 0) head_part_z_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(part, P, part_stride, b2, z, n);
}

void launch_init_state(const StepArgs *A, int n_sub, cudaStream_t s) {
    init_state_kernel<<<(n_sub + 255) / 256 + 1, 256, 0, s>>>(A);
}

void launch_compact(const StepArgs *A, cudaStream_t s, bool pdl) {
    launch_k(pdl, compact_kernel, dim3(1), dim3(1024), 0, s, A);
}

void launch_totals(const StepArgs *A, unsigned long long *out, int n_sub, cudaStream_t s) {
    int blocks = (n_sub + 255) / 256;
    if (blocks > 148) blocks = 148;
    if (blocks < 1) blocks = 1;
    totals_kernel<<<blocks, 256, 0, s>>>(A, out);
}

}  // namespace simnet
