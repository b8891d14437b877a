// gemm_simt.cu -- the FP32 form of the CNN's layers on CUDA cores (FFMA, no
// tensor cores): C[M,N] = act(A[M,K] * B[N,K]^T + bias).  A k=2/stride-2
// convolution over rows (2l, 2l+1) is this GEMM on the contiguous reshape of
// its input (Sec. 2.3); so is the FC layer on the flattened activations.
#include "common.cuh"
#include "kernels.cuh"

namespace simnet {

// 128 x BN tile, BK = 8, 256 threads; each thread owns an 8 x (BN/16) block of C.
// Shared tiles are stored K-major so the inner loop reads float4 runs of M and N.
// NO > 0: instead of storing C, fold FC2 (w2 [NO][N], NO in {2, 3, 22, 33}) into the epilogue and write
// per-column-block partial dot products C_part[blockIdx.y][row][0..NO).
template <int BN, int NO>
__global__ void __launch_bounds__(256) sgemm_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                    const float *__restrict__ bias, float *__restrict__ C,
                                                    const int32_t *__restrict__ n_active, int m_mult,
                                                    int m_cap, int N, int K, int relu,
                                                    const float *__restrict__ w2, int part_stride,
                                                    const float *__restrict__ R) {
    constexpr int BM = 128, BK = 8, TM = 8, TN = BN / 16;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int M = min(*n_active * m_mult, m_cap);
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    if (m0 >= M) return;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // loader coordinates: one float4 of A per thread, one of B per thread (BN=128) or half the threads (BN=64)
    const int lrow = tid >> 1, lk = (tid & 1) * 4;
    const bool a_ok = (m0 + lrow) < M;
    const bool b_ld = lrow < BN;
    const bool b_ok = b_ld && (n0 + lrow) < N;
    const float *Ap = A + (size_t)(m0 + lrow) * K + lk;
    const float *Bp = B + (size_t)(n0 + lrow) * K + lk;

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = 0.f;

    float4 ra = a_ok ? *reinterpret_cast<const float4 *>(Ap) : make_float4(0, 0, 0, 0);
    float4 rb = b_ok ? *reinterpret_cast<const float4 *>(Bp) : make_float4(0, 0, 0, 0);
    int buf = 0;
    As[0][lk + 0][lrow] = ra.x; As[0][lk + 1][lrow] = ra.y; As[0][lk + 2][lrow] = ra.z; As[0][lk + 3][lrow] = ra.w;
    if (b_ld) { Bs[0][lk + 0][lrow] = rb.x; Bs[0][lk + 1][lrow] = rb.y; Bs[0][lk + 2][lrow] = rb.z; Bs[0][lk + 3][lrow] = rb.w; }
    __syncthreads();

    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) {  // prefetch the next K slice into registers
            ra = a_ok ? *reinterpret_cast<const float4 *>(Ap + k0 + BK) : make_float4(0, 0, 0, 0);
            rb = b_ok ? *reinterpret_cast<const float4 *>(Bp + k0 + BK) : make_float4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < BK; k++) {
            float a[TM], b[TN];
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * TM]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * TM + 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
            for (int j = 0; j < TN; j += 4) {
                const float4 bv = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * TN + j]);
                b[j] = bv.x; b[j + 1] = bv.y; b[j + 2] = bv.z; b[j + 3] = bv.w;
            }
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            buf ^= 1;
            As[buf][lk + 0][lrow] = ra.x; As[buf][lk + 1][lrow] = ra.y; As[buf][lk + 2][lrow] = ra.z; As[buf][lk + 3][lrow] = ra.w;
            if (b_ld) { Bs[buf][lk + 0][lrow] = rb.x; Bs[buf][lk + 1][lrow] = rb.y; Bs[buf][lk + 2][lrow] = rb.z; Bs[buf][lk + 3][lrow] = rb.w; }
            __syncthreads();
        }
    }
    if constexpr (NO > 0) {
#pragma unroll
        for (int i = 0; i < TM; i++) {
            float p[NO];
#pragma unroll
            for (int o = 0; o < NO; o++) p[o] = 0.f;
#pragma unroll
            for (int j = 0; j < TN; j++) {
                const int col = n0 + tx * TN + j;
                float v = acc[i][j] + bias[col];
                if (relu) v = fmaxf(v, 0.f);
#pragma unroll
                for (int o = 0; o < NO; o++) p[o] = fmaf(v, w2[(size_t)o * N + col], p[o]);
            }
            // the 16 threads of a row group sit in one half-warp
#pragma unroll
            for (int o = 0; o < NO; o++)
#pragma unroll
                for (int d = 1; d < 16; d <<= 1) p[o] += __shfl_xor_sync(0xffffffffu, p[o], d);
            const int row = m0 + ty * TM + i;
            if (row < M) {
                float *dst = C + ((size_t)blockIdx.y * part_stride + row) * NO;
#pragma unroll
                for (int o = 0; o < NO; o++)
                    if (tx == (o & 15)) dst[o] = p[o];
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int row = m0 + ty * TM + i;
        if (row >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
            const int col = n0 + tx * TN + j;
            if (col >= N) continue;
            float4 v;
            v.x = acc[i][j] + bias[col];
            v.y = acc[i][j + 1] + bias[col + 1];
            v.z = acc[i][j + 2] + bias[col + 2];
            v.w = acc[i][j + 3] + bias[col + 3];
            if (R) {   // residual block: the shortcut, before the activation
                const float4 r = *reinterpret_cast<const float4 *>(R + (size_t)row * N + col);
                v.x += r.x; v.y += r.y; v.z += r.z; v.w += r.w;
            }
            if (relu) { v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f); }
            *reinterpret_cast<float4 *>(C + (size_t)row * N + col) = v;
        }
    }
}

void launch_gemm_f32(const float *A, const float *B, const float *bias, float *C, const int32_t *n_active,
                     int m_mult, int m_cap, int N, int K, int relu, cudaStream_t s, bool pdl, const float *R) {
    const unsigned gm = (unsigned)((m_cap + 127) / 128);
    if (gm == 0) return;
    if (N % 128 == 0)
        launch_k(pdl, sgemm_kernel<128, 0>, dim3(gm, N / 128), dim3(256), 0, s, A, B, bias, C, n_active, m_mult,
                 m_cap, N, K, relu, (const float *)nullptr, 0, R);
    else
        launch_k(pdl, sgemm_kernel<64, 0>, dim3(gm, (N + 63) / 64), dim3(256), 0, s, A, B, bias, C, n_active,
                 m_mult, m_cap, N, K, relu, (const float *)nullptr, 0, R);
}

int gemm_f32_part_blocks(int N) { return N % 128 == 0 ? N / 128 : (N + 63) / 64; }

template <int NO>
static void launch_part_no(const float *A, const float *B, const float *bias, const float *w2, float *part,
                           int part_stride, const int32_t *n_active, int m_mult, int m_cap, int N, int K, int relu,
                           cudaStream_t s, bool pdl) {
    const unsigned gm = (unsigned)((m_cap + 127) / 128);
    if (gm == 0) return;
    if (N % 128 == 0)
        launch_k(pdl, sgemm_kernel<128, NO>, dim3(gm, N / 128), dim3(256), 0, s, A, B, bias, part, n_active, m_mult,
                 m_cap, N, K, relu, w2, part_stride, (const float *)nullptr);
    else
        launch_k(pdl, sgemm_kernel<64, NO>, dim3(gm, (N + 63) / 64), dim3(256), 0, s, A, B, bias, part, n_active,
                 m_mult, m_cap, N, K, relu, w2, part_stride, (const float *)nullptr);
}

void launch_gemm_f32_part(const float *A, const float *B, const float *bias, const float *w2, float *part,
                          int part_stride, const int32_t *n_active, int m_mult, int m_cap, int N, int K, int relu,
                          int n_out, cudaStream_t s, bool pdl) {
    switch (n_out) {
        case 3: launch_part_no<3>(A, B, bias, w2, part, part_stride, n_active, m_mult, m_cap, N, K, relu, s, pdl); break;
        case 22: launch_part_no<22>(A, B, bias, w2, part, part_stride, n_active, m_mult, m_cap, N, K, relu, s, pdl); break;
        case 33: launch_part_no<33>(A, B, bias, w2, part, part_stride, n_active, m_mult, m_cap, N, K, relu, s, pdl); break;
        default: launch_part_no<2>(A, B, bias, w2, part, part_stride, n_active, m_mult, m_cap, N, K, relu, s, pdl); break;
    }
}

}  // namespace simnet
