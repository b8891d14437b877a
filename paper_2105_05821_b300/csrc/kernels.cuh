// kernels.cuh -- host-side launchers of libsimnet's kernels.
#pragma once
#include "common.cuh"

namespace simnet {

template <typename T>
void launch_gather(const StepArgs *A, T *X, int n_slots, int window, cudaStream_t s, bool pdl = false);
template <typename T> void launch_pack_x(const float *x, T *X, int64_t rows, cudaStream_t s);
// FC2 from P partial sums [P][part_stride][n_out] + queue update; writes the next step's rows of X.
template <typename T>
void launch_head_update(const StepArgs *A, const float *part, int P, int part_stride, const float *b2, T *X,
                        int n_slots, int n_out, cudaStream_t s, bool pdl = false);
// z [n][n_out] = h [n][H] * w2^T + b2 (w2 [n_out][H]).
void launch_head_z(const float *h, const float *w2, const float *b2, float *z, int n, int H, int n_out,
                   cudaStream_t s);
// z [n][n_out] = b2 + the sum of P partials [P][part_stride][n_out].
void launch_head_part_z(const float *part, int P, int part_stride, const float *b2, float *z, int n, int n_out,
                        cudaStream_t s);
void launch_init_state(const StepArgs *A, int n_sub, cudaStream_t s);
void launch_compact(const StepArgs *A, cudaStream_t s, bool pdl = false);
void launch_totals(const StepArgs *A, unsigned long long *out, int n_sub, cudaStream_t s);
void launch_channel_amax(const float *y, int64_t rows, int C, unsigned *out, cudaStream_t s);

// FP32 CUDA-core GEMM: C[M,N] = act(A[M,K] * B[N,K]^T + bias [+ R]), M = min(*n_active * m_mult, m_cap);
// R [M][N] (the shortcut of a residual block) or null.
void launch_gemm_f32(const float *A, const float *B, const float *bias, float *C, const int32_t *n_active,
                     int m_mult, int m_cap, int N, int K, int relu, cudaStream_t s, bool pdl = false,
                     const float *R = nullptr);
// The same with FC2 (w2 [n_out][N], n_out 2 or 22) folded into the epilogue:
// part [gemm_f32_part_blocks(N)][part_stride][n_out] float.
int gemm_f32_part_blocks(int N);
void launch_gemm_f32_part(const float *A, const float *B, const float *bias, const float *w2, float *part,
                          int part_stride, const int32_t *n_active, int m_mult, int m_cap, int N, int K, int relu,
                          int n_out, cudaStream_t s, bool pdl = false);

// FP32 weights of a context, for entry points defined outside simnet.cu.
struct CtxFp32View {
    int window = 0, hidden = 0, n_layers = 0, device = 0, n_out = 2;
    GemmLayer layer[kMaxGemm];
    const float *w2 = nullptr, *b2 = nullptr;
};
bool ctx_fp32_view(const simnet_ctx *c, CtxFp32View &v);
void ctx_set_error(simnet_ctx *c, const char *msg);

}  // namespace simnet
