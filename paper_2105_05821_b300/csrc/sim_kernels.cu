// sim_kernels.cu -- per-step simulation kernels: context gather (Sec. 2.2), the
// latency head and the processor-queue / curTick update (Sec. 3.2), the drain
// of Eq. 1 (Sec. 3.1), active-set compaction for uneven sub-traces (Sec. 3.3).
#include "common.cuh"
#include "kernels.cuh"
#include "sim_device.cuh"

namespace simnet {

// One warp per 32 consecutive rows (slot-major), staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(128) gather_kernel(const StepArgs *__restrict__ A, T *__restrict__ X,
                                                     int n_slots) {
    __shared__ __align__(16) uint8_t stg[4][32 * stage_row_bytes<T>()];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t total = (int64_t)n_slots * A->window;
    const int64_t row0 = ((int64_t)blockIdx.x * 4 + (threadIdx.x >> 5)) * 32;
    if (row0 >= total) return;
    gather_rows_warp<T>(A, X, row0, total, stg[threadIdx.x >> 5], threadIdx.x & 31);
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

// One warp per active slot (see head_update_warp); dynamic shared memory holds,
// per warp, 256 queue entries and 32 staged rows.
template <typename T, int NO>
__global__ void __launch_bounds__(256) head_update_kernel(const StepArgs *__restrict__ A,
                                                          const float *__restrict__ part, int P,
                                                          int part_stride, const float *__restrict__ b2,
                                                          T *__restrict__ X) {
    extern __shared__ __align__(16) uint8_t hsm[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int slot = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (slot >= *A->n_active) return;
    constexpr int PER = 256 * 8 + 32 * stage_row_bytes<T>();
    uint8_t *mine = hsm + w * PER;
    head_update_warp<T, NO>(A, slot, lane, part, P, part_stride, b2, X, reinterpret_cast<uint64_t *>(mine),
                            mine + 256 * 8);
}

// FC2 from partial dot products: z = b2 + sum of P partials (pre-softplus), one warp per row.
template <int NO>
__global__ void __launch_bounds__(256) head_part_z_kernel(const float *__restrict__ part, int P, int part_stride,
                                                          const float *__restrict__ b2, float *__restrict__ z,
                                                          int n) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float zr[NO];
    head_sum_warp<NO>(part, P, part_stride, row, b2, lane, zr);
#pragma unroll
    for (int o = 0; o < NO; o++)
        if (lane == o % 32) z[(size_t)row * NO + o] = zr[o];
}

// FC2 only (pre-softplus outputs, w2 [n_out][H]) for the CNN-only entry points:
// one warp per row, lanes over H, one output at a time.
__global__ void __launch_bounds__(256) head_z_kernel(const float *__restrict__ h, const float *__restrict__ w2,
                                                     const float *__restrict__ b2, float *__restrict__ z,
                                                     int n, int H, int n_out) {
    const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *hv = h + (size_t)row * H;
    for (int o = 0; o < n_out; o++) {
        float acc = 0.f;
        for (int j = lane; j < H; j += 32) acc = fmaf(hv[j], w2[(size_t)o * H + j], acc);
        acc = warp_sum(acc);
        if (lane == 0) z[(size_t)row * n_out + o] = acc + b2[o];
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
    if (A->mlen) {
        A->mstart[b] = 0;
        A->mlen[b] = 0;
    }
    A->evict[b] = 0;
    A->active[b] = b;
    A->cycles_out[b] = 0;
}

__global__ void __launch_bounds__(1024) compact_kernel(const StepArgs *__restrict__ A) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    compact_block(A);
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
    const int64_t total = (int64_t)n_slots * window;   // rows; 4 warps x 32 rows per block
    launch_k(pdl, gather_kernel<T>, dim3((unsigned)((total + 127) / 128)), dim3(128), 0, s, A, X, n_slots);
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

template <typename T, int NO>
static void launch_head_update_no(const StepArgs *A, const float *part, int P, int part_stride, const float *b2,
                                  T *X, int n_slots, cudaStream_t s, bool pdl) {
    const int64_t threads = (int64_t)n_slots * 32;
    const size_t smem = 8 * (256 * 8 + 32 * stage_row_bytes<T>());
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(head_update_kernel<T, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    launch_k(pdl, head_update_kernel<T, NO>, dim3((unsigned)((threads + 255) / 256)), dim3(256), smem, s, A, part,
             P, part_stride, b2, X);
}

template <typename T>
void launch_head_update(const StepArgs *A, const float *part, int P, int part_stride, const float *b2, T *X,
                        int n_slots, int n_out, cudaStream_t s, bool pdl) {
    switch (n_out) {
        case 3: launch_head_update_no<T, 3>(A, part, P, part_stride, b2, X, n_slots, s, pdl); break;
        case 22: launch_head_update_no<T, 22>(A, part, P, part_stride, b2, X, n_slots, s, pdl); break;
        case 33: launch_head_update_no<T, 33>(A, part, P, part_stride, b2, X, n_slots, s, pdl); break;
        default: launch_head_update_no<T, 2>(A, part, P, part_stride, b2, X, n_slots, s, pdl); break;
    }
}
template void launch_head_update<float>(const StepArgs *, const float *, int, int, const float *, float *, int, int,
                                        cudaStream_t, bool);
template void launch_head_update<__nv_bfloat16>(const StepArgs *, const float *, int, int, const float *,
                                                __nv_bfloat16 *, int, int, cudaStream_t, bool);
template void launch_head_update<__nv_fp8_e4m3>(const StepArgs *, const float *, int, int, const float *,
                                                __nv_fp8_e4m3 *, int, int, cudaStream_t, bool);

void launch_head_z(const float *h, const float *w2, const float *b2, float *z, int n, int H, int n_out,
                   cudaStream_t s) {
    const int64_t threads = (int64_t)n * 32;
    if (n > 0) head_z_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(h, w2, b2, z, n, H, n_out);
}

void launch_head_part_z(const float *part, int P, int part_stride, const float *b2, float *z, int n, int n_out,
                        cudaStream_t s) {
    const int64_t threads = (int64_t)n * 32;
    if (n <= 0) return;
    const unsigned g = (unsigned)((threads + 255) / 256);
    switch (n_out) {
        case 3: head_part_z_kernel<3><<<g, 256, 0, s>>>(part, P, part_stride, b2, z, n); break;
        case 22: head_part_z_kernel<22><<<g, 256, 0, s>>>(part, P, part_stride, b2, z, n); break;
        case 33: head_part_z_kernel<33><<<g, 256, 0, s>>>(part, P, part_stride, b2, z, n); break;
        default: head_part_z_kernel<2><<<g, 256, 0, s>>>(part, P, part_stride, b2, z, n); break;
    }
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
