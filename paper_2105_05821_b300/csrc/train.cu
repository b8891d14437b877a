// train.cu -- training the latency predictor (Sec. 2.4): windows labelled by a
// timing model, the CNN forward with saved activations, hand-written backward
// kernels for the loss, FC and k=2/stride-2 conv layers, and Adam.
//
// FP32 contexts run every GEMM on one strided FP32 kernel (CUDA cores) covering
// the three forms a layer needs: Y = A W^T (forward), dA = dY W (input
// gradient) and dW = dY^T A (weight gradient, split over rows with atomic
// accumulation).  BF16 contexts (autocast numerics: BF16 operands, FP32 sums)
// run the same three forms on the tcgen05 tensor cores (train_tc.cu), with the
// windows, saved activations and gradients of the conv outputs in BF16; FC2, the
// loss and the FC1 output stay FP32.  Master weights, moments and weight
// gradients are FP32 in both; one Adam kernel updates every parameter and
// refreshes a BF16 context's BF16 weight copies.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "sim_device.cuh"

namespace simnet {
namespace {

// ------------------------------------------------------------------ windows
// X [n][W][64] (FP32 or BF16; optionally also x50 [n][W][50] FP32): row 0 =
// instruction i, row r = instruction i-r while i-r >= ctx_begin[i], residence
// fetch[i-1] - fetch[i-r].  Every value is k / 2^m with few bits: exact in BF16.
template <typename T>
__global__ void window_gather_kernel(const uint32_t *__restrict__ rec, const int64_t *__restrict__ fetch,
                                     const uint8_t *__restrict__ e_label, const int64_t *__restrict__ ctx_begin,
                                     const int64_t *__restrict__ idx, int n, int W, T *__restrict__ X,
                                     float *__restrict__ x50) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * W * 16) return;
    const int chunk = (int)(gid & 15);
    const int64_t rowid = gid >> 4;
    const int r = (int)(rowid % W);
    const int s = (int)(rowid / W);
    const int64_t i = idx[s];
    const uint32_t cur = rec[i];
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r == 0) {
        for (int j = 0; j < 4; j++) v[j] = feature(chunk * 4 + j, cur, cur, false, 0, 0, 0);
    } else if (i - r >= ctx_begin[i]) {
        const int64_t jj = i - r;
        const int64_t now = i > 0 ? fetch[i - 1] : 0;
        const int64_t res = now - fetch[jj];
        const int32_t res32 = (int32_t)(res > 4095 ? 4095 : res);
        for (int j = 0; j < 4; j++) v[j] = feature(chunk * 4 + j, rec[jj], cur, true, res32, e_label[jj], 0);
    }
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(X + rowid * kNFP + chunk * 4) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
        *reinterpret_cast<uint2 *>(X + rowid * kNFP + chunk * 4) =
            make_uint2(*reinterpret_cast<uint32_t *>(&p0), *reinterpret_cast<uint32_t *>(&p1));
    }
    if (x50)
        for (int j = 0; j < 4; j++)
            if (chunk * 4 + j < kNF) x50[rowid * kNF + chunk * 4 + j] = v[j];
}

// The same rows for the training step, one thread per row: the row's 64 channels
// built whole by the simulator's row writer (the values `feature` gives).
template <typename T>
__global__ void window_rows_kernel(const uint32_t *__restrict__ rec, const int64_t *__restrict__ fetch,
                                   const uint8_t *__restrict__ e_label, const int64_t *__restrict__ ctx_begin,
                                   const int64_t *__restrict__ idx, int n, int W, T *__restrict__ X) {
    const int64_t rowid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rowid >= (int64_t)n * W) return;
    const int r = (int)(rowid % W);
    const int64_t i = idx[rowid / W];
    const uint32_t cur = rec[i];
    T *dst = X + rowid * kNFP;
    if (r == 0) {
        write_row<T>(dst, cur, cur, false, 0, 0u, 0u);
    } else if (i - r >= ctx_begin[i]) {
        const int64_t jj = i - r;
        const int64_t res = (i > 0 ? fetch[i - 1] : 0) - fetch[jj];
        write_row<T>(dst, rec[jj], cur, true, (int32_t)(res > 4095 ? 4095 : res), e_label[jj], 0u);
    } else {
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
        for (int k = 0; k < kNFP * (int)sizeof(T) / 16; k++) d4[k] = make_uint4(0, 0, 0, 0);
    }
}

// ------------------------------------------------------------------ strided GEMM
// C(m, n) = sum_k A(m, k) B(k, n), A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn].
// K is split over gridDim.z; with `accumulate` every split atomically adds
// into C (which the caller zeroes), else the single split stores C, + bias, ReLU.
template <bool ROUND>
__global__ void __launch_bounds__(256) gemm_strided_kernel(const float *__restrict__ A, int64_t sam, int64_t sak,
                                                           const float *__restrict__ B, int64_t sbk, int64_t sbn,
                                                           float *__restrict__ C, int64_t ldc, int M, int N, int K,
                                                           int k_chunk, const float *__restrict__ bias, int relu,
                                                           int accumulate) {
    constexpr int T = 64, BK = 16;
    __shared__ float As[BK][T + 4], Bs[BK][T + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * T, n0 = blockIdx.x * T;
    const int k_lo = blockIdx.z * k_chunk, k_hi = min(K, k_lo + k_chunk);
    const bool a_kfast = sak == 1, b_nfast = sbn == 1;
    float acc[4][4] = {};
    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int e = tid + 256 * q;
            int mm, kk;
            if (a_kfast) { kk = e & 15; mm = e >> 4; } else { mm = e & 63; kk = e >> 6; }
            const int gm = m0 + mm, gk = k0 + kk;
            float a = (gm < M && gk < k_hi) ? A[gm * sam + gk * sak] : 0.f;
            if (ROUND) a = __bfloat162float(__float2bfloat16_rn(a));
            As[kk][mm] = a;
            int nn, kb;
            if (b_nfast) { nn = e & 63; kb = e >> 6; } else { kb = e & 15; nn = e >> 4; }
            const int gn = n0 + nn, gkb = k0 + kb;
            float b = (gn < N && gkb < k_hi) ? B[gkb * sbk + gn * sbn] : 0.f;
            if (ROUND) b = __bfloat162float(__float2bfloat16_rn(b));
            Bs[kb][nn] = b;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; k++) {
            const float4 a4 = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            if (accumulate) {
                atomicAdd(C + (int64_t)m * ldc + n, acc[i][j]);
            } else {
                float v = acc[i][j] + (bias ? bias[n] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                C[(int64_t)m * ldc + n] = v;
            }
        }
    }
}

// The same product on 128 x TN tiles (TN = 64 or 128), each thread 8 x TN/16
// outputs, the next K slice loaded into registers while the current one is
// multiplied (for products with enough 128-row tiles to fill the GPU).
template <bool ROUND, int TN>
__global__ void __launch_bounds__(256) gemm_strided_tile_kernel(const float *__restrict__ A, int64_t sam, int64_t sak,
                                                                const float *__restrict__ B, int64_t sbk,
                                                                int64_t sbn, float *__restrict__ C, int64_t ldc, int M,
                                                                int N, int K, int k_chunk,
                                                                const float *__restrict__ bias, int relu,
                                                                int accumulate) {
    constexpr int TM = 128, BK = 16, NA = TM * BK / 256, NB = TN * BK / 256, CN = TN / 16;
    __shared__ __align__(16) float As[BK][TM + 4];
    __shared__ __align__(16) float Bs[BK][TN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int k_lo = blockIdx.z * k_chunk, k_hi = min(K, k_lo + k_chunk);
    const bool a_kfast = sak == 1, b_nfast = sbn == 1;
    float ra[NA], rb[NB];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < NA; q++) {
            const int e = tid + 256 * q;
            int mm, kk;
            if (a_kfast) { kk = e & (BK - 1); mm = e / BK; } else { mm = e & (TM - 1); kk = e / TM; }
            const int gm = m0 + mm, gk = k0 + kk;
            float v = (gm < M && gk < k_hi) ? A[(int64_t)gm * sam + (int64_t)gk * sak] : 0.f;
            if (ROUND) v = __bfloat162float(__float2bfloat16_rn(v));
            ra[q] = v;
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int e = tid + 256 * q;
            int nn, kb;
            if (b_nfast) { nn = e & (TN - 1); kb = e / TN; } else { kb = e & (BK - 1); nn = e / BK; }
            const int gn = n0 + nn, gk = k0 + kb;
            float v = (gn < N && gk < k_hi) ? B[(int64_t)gk * sbk + (int64_t)gn * sbn] : 0.f;
            if (ROUND) v = __bfloat162float(__float2bfloat16_rn(v));
            rb[q] = v;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int q = 0; q < NA; q++) {
            const int e = tid + 256 * q;
            if (a_kfast) As[e & (BK - 1)][e / BK] = ra[q];
            else As[e / TM][e & (TM - 1)] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int e = tid + 256 * q;
            if (b_nfast) Bs[e / TN][e & (TN - 1)] = rb[q];
            else Bs[e & (BK - 1)][e / BK] = rb[q];
        }
    };
    float acc[8][CN] = {};
    if (k_lo < k_hi) load(k_lo);
    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
        store();
        __syncthreads();
        if (k0 + BK < k_hi) load(k0 + BK);   // the next slice's global loads overlap this slice's FMAs
#pragma unroll
        for (int k = 0; k < BK; k++) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][ty * 8 + 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[CN];
#pragma unroll
            for (int j4 = 0; j4 < CN / 4; j4++) {
                const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[k][tx * CN + 4 * j4]);
                b[4 * j4] = b4.x;
                b[4 * j4 + 1] = b4.y;
                b[4 * j4 + 2] = b4.z;
                b[4 * j4 + 3] = b4.w;
            }
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < CN; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int m = m0 + ty * 8 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < CN; j++) {
            const int n = n0 + tx * CN + j;
            if (n >= N) continue;
            if (accumulate) {
                atomicAdd(C + (int64_t)m * ldc + n, acc[i][j]);
            } else {
                float v = acc[i][j] + (bias ? bias[n] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                C[(int64_t)m * ldc + n] = v;
            }
        }
    }
}

// C(m, n) = (relu) (C(m, n) + bias[n]): the epilogue of a product whose K was split
__global__ void bias_relu_kernel(float *__restrict__ C, int64_t ldc, int M, int N, const float *__restrict__ bias,
                                 int relu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int m = (int)(i / N), n = (int)(i % N);
    float v = C[(int64_t)m * ldc + n] + (bias ? bias[n] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    C[(int64_t)m * ldc + n] = v;
}

// ------------------------------------------------------------------ elementwise
__global__ void relu_mask_kernel(float *__restrict__ d, const float *__restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(y[i] > 0.f)) d[i] = 0.f;
}

// out[c] += sum over rows of d[r][c]
__global__ void colsum_kernel(const float *__restrict__ d, int64_t rows, int C, float *__restrict__ out) {
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) s += d[r * C + c];
    atomicAdd(out + c, s);
}

// z -> softplus; loss += (y - t)^2 / (2n) with t the label clamped to [0, 255];
// dz = (y - t) / n * sigmoid(z) (1 above the softplus threshold), times *gs when
// given.  The label of row r is labels[2 idx[r] + k] (labels[2 r + k] without
// idx); dz may be null (loss only).
__global__ void mse_softplus_kernel(const float *__restrict__ z, const uint8_t *__restrict__ labels,
                                    const int64_t *__restrict__ idx, int n, float *__restrict__ dz,
                                    double *__restrict__ loss, const float *__restrict__ gs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < 2 * n) {
        const int r = i >> 1, k = i & 1;
        const float x = z[i];
        const float y = x > 20.f ? x : log1pf(expf(x));
        const float t = (float)labels[2 * (idx ? idx[r] : (int64_t)r) + k];
        const float diff = y - t;
        const float sg = x > 20.f ? 1.f : 1.f / (1.f + expf(-x));
        if (dz) dz[i] = diff / (float)n * sg * (gs ? *gs : 1.f);
        l = (double)diff * diff / (2.0 * n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// Hybrid head (Sec. 2.3), one thread per (window r, latency k): z holds 22
// outputs per window, the ten class logits of latency k at 11k..11k+9 and its
// regression output at 11k+10.  loss += (CE + (softplus(z_v) - t)^2) / (2n) with
// CE = logsumexp(logits) - logit[min(t, 9)]; dz of the logits = (softmax - onehot)
// / (2n), of the value (softplus(z_v) - t) / n * sigmoid(z_v); labels, idx, gs and a
// null dz as for mse_softplus_kernel.
__global__ void hybrid_loss_kernel(const float *__restrict__ z, const uint8_t *__restrict__ labels,
                                   const int64_t *__restrict__ idx, int n, float *__restrict__ dz,
                                   double *__restrict__ loss, const float *__restrict__ gs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < 2 * n) {
        const int r = i >> 1, k = i & 1;
        const float *lg = z + (size_t)r * 22 + 11 * k;
        const int t = labels[2 * (idx ? idx[r] : (int64_t)r) + k];
        const int cls = t > 8 ? 9 : t;
        float mx = lg[0];
        for (int j = 1; j < 10; j++) mx = fmaxf(mx, lg[j]);
        float se = 0.f;
        for (int j = 0; j < 10; j++) se += expf(lg[j] - mx);
        const float x = lg[10];
        const float y = x > 20.f ? x : log1pf(expf(x));
        const float diff = y - (float)t;
        const float sg = x > 20.f ? 1.f : 1.f / (1.f + expf(-x));
        if (dz) {
            float *dl = dz + (size_t)r * 22 + 11 * k;
            const float g = gs ? *gs : 1.f, inv2n = 1.f / (2.f * (float)n);
            for (int j = 0; j < 10; j++) dl[j] = (expf(lg[j] - mx) / se - (j == cls ? 1.f : 0.f)) * inv2n * g;
            dl[10] = diff / (float)n * sg * g;
        }
        const double ce = (double)mx + log((double)se) - (double)lg[cls];
        l = (ce + (double)diff * diff) / (2.0 * n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// Adam over every parameter array of the CNN in one launch: segment k holds
// parameters [start[k], start[k+1]) of the concatenation; a BF16 context's
// weight segments also rewrite their BF16 copy.
struct AdamSeg {
    float *th, *m, *v;
    const float *g;
    __nv_bfloat16 *shadow;   // or null
};
constexpr int kAdamSegs = 2 * kMaxGemm + 2;
struct AdamTable {
    AdamSeg seg[kAdamSegs];
    int64_t start[kAdamSegs + 1];
    int nseg;
};

__global__ void adam_multi_kernel(const __grid_constant__ AdamTable T, float lr, float b1, float b2, float eps,
                                  float c1, float c2) {
    const int64_t total = T.start[T.nseg];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (i >= T.start[k + 1]) k++;
        const AdamSeg &S = T.seg[k];
        const int64_t j = i - T.start[k];
        const float gi = S.g[j];
        const float mi = b1 * S.m[j] + (1.f - b1) * gi;
        const float vi = b2 * S.v[j] + (1.f - b2) * gi * gi;
        S.m[j] = mi;
        S.v[j] = vi;
        const float th = S.th[j] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        S.th[j] = th;
        if (S.shadow) S.shadow[j] = __float2bfloat16_rn(th);
    }
}

// ------------------------------------------------------------------ BF16 training (tensor cores)
// FC2 backward for a block of 32 windows, one thread per FC1 neuron h:
// gw2[o][h] += sum_r dz[r][o] H[r][h], gb2[o] += sum_r dz[r][o], and
// dH[r][h] = (sum_o dz[r][o] w2[o][h]) where H[r][h] > 0 (BF16, the next
// GEMM's operand), whose FP32 column sums are FC1's bias gradient gb1[h].
template <int NO>
__global__ void __launch_bounds__(256) head_bwd_kernel(const float *__restrict__ Hh, const float *__restrict__ dz,
                                                       const float *__restrict__ w2, int n, int H,
                                                       __nv_bfloat16 *__restrict__ dH, float *__restrict__ gw2,
                                                       float *__restrict__ gb2, float *__restrict__ gb1) {
    constexpr int RB = 32;
    __shared__ float s_dz[RB][NO];
    const int r0 = blockIdx.x * RB, rn = min(RB, n - r0);
    for (int i = threadIdx.x; i < RB * NO; i += blockDim.x) {
        const int r = i / NO, o = i % NO;
        s_dz[r][o] = r < rn ? dz[(size_t)(r0 + r) * NO + o] : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < NO) {
        float sum = 0.f;
        for (int r = 0; r < rn; r++) sum += s_dz[r][threadIdx.x];
        atomicAdd(&gb2[threadIdx.x], sum);
    }
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        float w[NO], g[NO];
#pragma unroll
        for (int o = 0; o < NO; o++) {
            w[o] = w2[(size_t)o * H + h];
            g[o] = 0.f;
        }
        float gb = 0.f;
        for (int r = 0; r < rn; r++) {
            const float hv = Hh[(size_t)(r0 + r) * H + h];
            float d = 0.f;
#pragma unroll
            for (int o = 0; o < NO; o++) {
                g[o] = fmaf(s_dz[r][o], hv, g[o]);
                d = fmaf(s_dz[r][o], w[o], d);
            }
            d = hv > 0.f ? d : 0.f;
            dH[(size_t)(r0 + r) * H + h] = __float2bfloat16_rn(d);
            gb += d;
        }
#pragma unroll
        for (int o = 0; o < NO; o++) atomicAdd(&gw2[(size_t)o * H + h], g[o]);
        atomicAdd(&gb1[h], gb);
    }
}

// Column sums out[c] = sum over rows of d[r][c] in two passes with no atomics:
// block g sums its share of the rows into part[g][c], then one thread per column
// adds the blocks' sums.  In a block a thread takes one 16-byte column vector
// (V = 8 BF16 or 4 FP32 columns) of every rpb-th row, four rows in flight, and
// the block adds its rpb row lanes in a fixed order through shared memory (the
// sums do not depend on scheduling).  The C columns are a row's first C of ld
// (the caller splits wider rows); C a multiple of V, at most 512; threads past
// the last whole row lane stay idle.
constexpr int kColBlocks = 2 * 148;
template <typename T>
__global__ void __launch_bounds__(256) colsum_part_kernel(const T *__restrict__ d, int64_t rows, int C, int ld,
                                                          float *__restrict__ part) {
    constexpr int V = 16 / (int)sizeof(T);
    __shared__ float sh[256 * V];   // [row lane][C]: rpb * C = 256 * V floats
    const int CV = C / V, cv = threadIdx.x % CV, rl = threadIdx.x / CV, rpb = blockDim.x / CV;
    const bool on = rl < rpb;
    float acc[V];
#pragma unroll
    for (int k = 0; k < V; k++) acc[k] = 0.f;
    auto add = [&](const uint4 &u) {
        if constexpr (sizeof(T) == 4) {
            acc[0] += __uint_as_float(u.x);
            acc[1] += __uint_as_float(u.y);
            acc[2] += __uint_as_float(u.z);
            acc[3] += __uint_as_float(u.w);
        } else {
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                // BF16 pair to FP32: each value's 16 bits as the high half of a word
                acc[2 * k] += __uint_as_float(w[k] << 16);
                acc[2 * k + 1] += __uint_as_float(w[k] & 0xffff0000u);
            }
        }
    };
    const uint4 *base = reinterpret_cast<const uint4 *>(d) + cv;
    const int64_t LV = ld / V;   // 16-byte vectors a row
    const int64_t step = (int64_t)gridDim.x * rpb;
    int64_t r = on ? (int64_t)blockIdx.x * rpb + rl : rows;
    for (; r + 3 * step < rows; r += 4 * step) {
        const uint4 u0 = base[r * LV], u1 = base[(r + step) * LV];
        const uint4 u2 = base[(r + 2 * step) * LV], u3 = base[(r + 3 * step) * LV];
        add(u0);
        add(u1);
        add(u2);
        add(u3);
    }
    for (; r < rows; r += step) add(base[r * LV]);
    if (on)
#pragma unroll
        for (int k = 0; k < V; k++) sh[rl * C + cv * V + k] = acc[k];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float t = 0.f;
        for (int q = 0; q < rpb; q++) t += sh[q * C + c];
        part[(size_t)blockIdx.x * C + c] = t;
    }
}

// A block takes 32 columns; its 8 warps sum every 8th block's sums (four loads in
// flight each), then one warp adds the 8.
__global__ void __launch_bounds__(256) colsum_final_kernel(const float *__restrict__ part, int G, int C,
                                                           float *__restrict__ out) {
    __shared__ float sh[8][33];
    const int e = threadIdx.x & 31, w = threadIdx.x >> 5, c = blockIdx.x * 32 + e;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (c < C) {
        int g = w;
        for (; g + 24 < G; g += 32) {
            s0 += part[(size_t)g * C + c];
            s1 += part[(size_t)(g + 8) * C + c];
            s2 += part[(size_t)(g + 16) * C + c];
            s3 += part[(size_t)(g + 24) * C + c];
        }
        for (; g < G; g += 8) s0 += part[(size_t)g * C + c];
    }
    sh[w][e] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (w == 0 && c < C) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; q++) t += sh[q][e];
        out[c] = t;
    }
}

__global__ void loss_to_float_kernel(const double *__restrict__ l, float *__restrict__ out) { *out = (float)*l; }

__global__ void to_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// Canonical PyTorch layout <-> GEMM layout of one layer's weights.
// conv: canonical [co][ci][t] <-> gemm [co][t*cin_pad + ci] (ci < cin)
// fc1:  canonical [h][ch*Ln + r] <-> gemm [h][r*C + ch]
__global__ void relayout_kernel(const float *__restrict__ src, float *__restrict__ dst, int is_conv, int rows,
                                int a, int b, int cin_pad, int to_gemm) {
    // conv: a = cin, b = 2 taps; fc1: a = C, b = Ln.  One thread per canonical element.
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)a * b;
    if (i >= (int64_t)rows * per) return;
    const int64_t row = i / per, rem = i % per;
    const int x = (int)(rem / b), y = (int)(rem % b);
    int64_t g;
    if (is_conv) g = row * (2 * cin_pad) + (int64_t)y * cin_pad + x;   // x = ci, y = t
    else g = row * per + (int64_t)y * a + x;                             // x = ch, y = r
    if (to_gemm) dst[g] = src[i];
    else dst[i] = src[g];
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace simnet

using namespace simnet;

template <int TN>
static void gemm_tile(bool round, const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbk, int64_t sbn,
                      float *C, int64_t ldc, int M, int N, int K, const float *bias, int relu, bool accumulate,
                      cudaStream_t s) {
    int splits = 1, chunk = K;
    if (accumulate) {
        const int tiles = ((M + 127) / 128) * ((N + TN - 1) / TN);
        splits = std::max(1, std::min((K + 255) / 256, 4 * 148 / std::max(tiles, 1)));
        chunk = ((K + splits - 1) / splits + 15) / 16 * 16;
        splits = (K + chunk - 1) / chunk;
    }
    dim3 g((N + TN - 1) / TN, (M + 127) / 128, splits);
    if (round)
        gemm_strided_tile_kernel<true, TN><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, chunk, bias,
                                                             relu, accumulate);
    else
        gemm_strided_tile_kernel<false, TN><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, chunk, bias,
                                                              relu, accumulate);
}

static void gemm(bool round, const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbk, int64_t sbn,
                 float *C, int64_t ldc, int M, int N, int K, const float *bias, int relu, bool accumulate,
                 cudaStream_t s) {
    // 128-row tiles when they alone fill the GPU twice over (the products over the
    // windows' rows); a product with few output tiles and a long K splits K
    // instead (atomically summed into C, then bias and ReLU)
    const int TN = N >= 128 ? 128 : 64;
    const int tiles128 = ((M + 127) / 128) * ((N + TN - 1) / TN), tiles64 = ((M + 63) / 64) * ((N + 63) / 64);
    if (M >= 128 && N >= 64 && (accumulate || tiles128 >= 2 * 148)) {
        if (TN == 128) gemm_tile<128>(round, A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, bias, relu, accumulate, s);
        else gemm_tile<64>(round, A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, bias, relu, accumulate, s);
        return;
    }
    if (!accumulate && tiles64 < 2 * 148 && K >= 512) {
        const int splits = std::min(K / 256, (4 * 148 + tiles64 - 1) / tiles64);
        const int chunk = ((K + splits - 1) / splits + 15) / 16 * 16;
        cudaMemset2DAsync(C, (size_t)ldc * sizeof(float), 0, (size_t)N * sizeof(float), (size_t)M, s);
        dim3 g((N + 63) / 64, (M + 63) / 64, (K + chunk - 1) / chunk);
        if (round)
            gemm_strided_kernel<true><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, chunk, nullptr, 0, 1);
        else
            gemm_strided_kernel<false><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, chunk, nullptr, 0, 1);
        if (bias || relu)
            bias_relu_kernel<<<(int)(((int64_t)M * N + 255) / 256), 256, 0, s>>>(C, ldc, M, N, bias, relu);
        return;
    }
    int splits = 1, chunk = K;
    if (accumulate) {  // long reductions (weight gradients): split the rows over blocks
        const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
        splits = std::max(1, std::min((K + 255) / 256, 4 * 148 / std::max(tiles, 1)));
        chunk = ((K + splits - 1) / splits + 15) / 16 * 16;
        splits = (K + chunk - 1) / chunk;
    }
    dim3 g((N + 63) / 64, (M + 63) / 64, splits);
    if (round)
        gemm_strided_kernel<true><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, chunk, bias, relu,
                                                    accumulate);
    else
        gemm_strided_kernel<false><<<g, 256, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, chunk, bias, relu,
                                                     accumulate);
}

static int64_t layer_rows(const simnet_ctx *c, int l, int n) { return (int64_t)n * c->layer[l].m_mult; }

// Tensor-core training: BF16 contexts.
static bool train_on_tc(const simnet_ctx *c) { return c->cfg.precision == SIMNET_BF16; }

// Allocate training buffers for n windows (and master-weight bookkeeping once).
simnet_status ensure_train(simnet_ctx *c, int n) {
    TrainState &t = c->tr;
    const simnet_config &k = c->cfg;
    if (!t.ready) {
        for (int l = 0; l < c->n_layers; l++) {
            const GemmLayer &g = c->layer[l];
            const size_t wn = (size_t)g.N * g.K;
            CK(cudaMalloc(&t.gW[l], wn * 4));
            CK(cudaMalloc(&t.mW[l], wn * 4));
            CK(cudaMalloc(&t.vW[l], wn * 4));
            CK(cudaMalloc(&t.gb[l], (size_t)g.N * 4));
            CK(cudaMalloc(&t.mb[l], (size_t)g.N * 4));
            CK(cudaMalloc(&t.vb[l], (size_t)g.N * 4));
            CK(cudaMemset(t.mW[l], 0, wn * 4));
            CK(cudaMemset(t.vW[l], 0, wn * 4));
            CK(cudaMemset(t.mb[l], 0, (size_t)g.N * 4));
            CK(cudaMemset(t.vb[l], 0, (size_t)g.N * 4));
        }
        const size_t h2 = (size_t)c->n_out * k.fc_hidden, b2n = (size_t)c->n_out * 4;
        CK(cudaMalloc(&t.gw2, h2 * 4));
        CK(cudaMalloc(&t.mw2, h2 * 4));
        CK(cudaMalloc(&t.vw2, h2 * 4));
        CK(cudaMalloc(&t.gb2, b2n));
        CK(cudaMalloc(&t.mb2, b2n));
        CK(cudaMalloc(&t.vb2, b2n));
        CK(cudaMemset(t.mw2, 0, h2 * 4));
        CK(cudaMemset(t.vw2, 0, h2 * 4));
        CK(cudaMemset(t.mb2, 0, b2n));
        CK(cudaMemset(t.vb2, 0, b2n));
        CK(cudaMalloc(&t.loss, sizeof(double)));
        CK(cudaMalloc(&t.colpart, (size_t)kColBlocks * 512 * sizeof(float)));
        t.ready = true;
    }
    if (n <= t.n_cap) return SIMNET_OK;
    CK(cudaDeviceSynchronize());
    void *old[] = {t.X, t.dA, t.dB, t.z, t.dz, t.Xb, t.dHb, t.dYb[0], t.dYb[1]};
    for (void *q : old)
        if (q) cudaFree(q);
    t.X = t.dA = t.dB = t.z = t.dz = nullptr;
    t.Xb = t.dHb = t.dYb[0] = t.dYb[1] = nullptr;
    for (int l = 0; l < c->n_layers; l++) {
        if (t.Y[l]) cudaFree(t.Y[l]);
        if (t.Yb[l]) cudaFree(t.Yb[l]);
        t.Y[l] = nullptr;
        t.Yb[l] = nullptr;
    }
    t.plan_n = -1;
    const int L = c->n_layers - 1;   // conv layers; layer L is FC1
    size_t big = 0;
    for (int l = 0; l < L; l++) big = std::max(big, (size_t)layer_rows(c, l, n) * c->layer[l].N);
    if (train_on_tc(c)) {
        CK(cudaMalloc(&t.Xb, (size_t)n * k.window * kNFP * 2));
        for (int l = 0; l < L; l++) CK(cudaMalloc(&t.Yb[l], (size_t)layer_rows(c, l, n) * c->layer[l].N * 2));
        CK(cudaMalloc(&t.Y[L], (size_t)n * k.fc_hidden * 4));   // FC1 output, FP32
        CK(cudaMalloc(&t.dHb, (size_t)n * k.fc_hidden * 2));
        CK(cudaMalloc(&t.dYb[0], std::max(big, (size_t)1) * 2));
        CK(cudaMalloc(&t.dYb[1], std::max(big, (size_t)1) * 2));
    } else {
        CK(cudaMalloc(&t.X, (size_t)n * k.window * kNFP * 4));
        size_t bigf = (size_t)n * k.window * kNFP;
        for (int l = 0; l < c->n_layers; l++) {
            const size_t e = (size_t)layer_rows(c, l, n) * c->layer[l].N;
            CK(cudaMalloc(&t.Y[l], e * 4));
            bigf = std::max(bigf, e);
        }
        CK(cudaMalloc(&t.dA, bigf * 4));
        CK(cudaMalloc(&t.dB, bigf * 4));
    }
    CK(cudaMalloc(&t.z, (size_t)n * c->n_out * 4));
    CK(cudaMalloc(&t.dz, (size_t)n * c->n_out * 4));
    t.n_cap = n;
    return SIMNET_OK;
}

// Device training: FP32 or BF16 contexts of plain conv layers (residual blocks
// have no backward pass in this library).
static bool train_precision_ok(const simnet_ctx *c) {
    return (c->cfg.precision == SIMNET_FP32 || c->cfg.precision == SIMNET_BF16) && !c->residual;
}

// The tensor-core GEMMs of a step over n windows (built when n changes).  Layer l
// reads A_l = the packed windows (l = 0) or layer l-1's output, viewed as
// [n * m_mult_l][K_l] (row pairs of a conv layer, the flatten for FC1).
static simnet_status tc_plans(simnet_ctx *c, int n) {
    TrainState &t = c->tr;
    if (t.plan_n == n) return SIMNET_OK;
    const int L = c->n_layers - 1, H = c->cfg.fc_hidden;
    std::string why;
    for (int l = 0; l <= L; l++) {
        const GemmLayer &g = c->layer[l];
        const int M = (int)layer_rows(c, l, n);
        const void *A = l == 0 ? (const void *)t.Xb : (const void *)t.Yb[l - 1];
        const void *dY = l == L ? (const void *)t.dHb : (const void *)t.dYb[l & 1];
        bool ok = make_tg_plan(t.fwd[l], l == L ? TG_FWD_F32 : TG_FWD_BF16, A, false, c->Wl[l], false, M, g.N, g.K,
                               l == L ? (void *)t.Y[L] : (void *)t.Yb[l], g.N, c->bias[l], nullptr, why);
        // weight gradient, stored transposed by the epilogue: rows = K (A's columns), columns = N
        ok = ok && make_tg_plan(t.wgrad[l], TG_WGRAD, A, true, dY, true, g.K, g.N, M, t.gW[l], g.K, nullptr, nullptr,
                                why);
        if (ok && l > 0)   // input gradient into layer l-1's output, masked by its ReLU
            ok = make_tg_plan(t.dgrad[l], TG_DGRAD, dY, false, c->Wl[l], true, M, g.K, g.N,
                              (void *)t.dYb[(l - 1) & 1], 0, nullptr, (const void *)t.Yb[l - 1], why);
        if (!ok) return fail(c, SIMNET_EUNSUPPORTED, "tensor-core training, layer %d: %s", l, why.c_str());
    }
    (void)H;
    // split scratch of the weight gradients and of FC1's forward (one GEMM at a time: one buffer)
    size_t need = 0;
    for (int l = 0; l <= L; l++) need = std::max({need, tg_part_floats(t.wgrad[l]), tg_part_floats(t.fwd[l])});
    if (need > t.wpart_cap) {
        CK(cudaDeviceSynchronize());
        if (t.wpart) cudaFree(t.wpart);
        t.wpart = nullptr;
        t.wpart_cap = 0;
        CK(cudaMalloc(&t.wpart, need * sizeof(float)));
        t.wpart_cap = need;
    }
    for (int l = 0; l <= L; l++) t.wgrad[l].part = t.fwd[l].part = t.wpart;
    t.plan_n = n;
    return SIMNET_OK;
}

// Forward over the packed windows: every layer's output kept; z = FC2.
static simnet_status train_forward_enqueue(simnet_ctx *c, int n, cudaStream_t s) {
    TrainState &t = c->tr;
    if (train_on_tc(c)) {
        simnet_status st = tc_plans(c, n);
        if (st != SIMNET_OK) return st;
        for (int l = 0; l < c->n_layers; l++) launch_tg(t.fwd[l], c->cfg.spin_limit_ns, c->status, s);
    } else {
        const float *in = t.X;
        for (int l = 0; l < c->n_layers; l++) {
            const GemmLayer &g = c->layer[l];
            const int R = (int)layer_rows(c, l, n);
            gemm(false, in, g.K, 1, c->W32[l], 1, g.K, t.Y[l], g.N, R, g.N, g.K, c->bias[l], 1, false, s);
            in = t.Y[l];
        }
    }
    launch_head_z(t.Y[c->n_layers - 1], c->w2, c->b2, t.z, n, c->cfg.fc_hidden, c->n_out, s);
    t.n_last = n;
    return SIMNET_OK;
}

static void launch_head_bwd(const float *Hh, const float *dz, const float *w2, int n, int H, int no,
                            __nv_bfloat16 *dH, float *gw2, float *gb2, float *gb1, cudaStream_t s) {
    const unsigned g = (unsigned)((n + 31) / 32);
    switch (no) {
        case 3: head_bwd_kernel<3><<<g, 256, 0, s>>>(Hh, dz, w2, n, H, dH, gw2, gb2, gb1); break;
        case 22: head_bwd_kernel<22><<<g, 256, 0, s>>>(Hh, dz, w2, n, H, dH, gw2, gb2, gb1); break;
        case 33: head_bwd_kernel<33><<<g, 256, 0, s>>>(Hh, dz, w2, n, H, dH, gw2, gb2, gb1); break;
        default: head_bwd_kernel<2><<<g, 256, 0, s>>>(Hh, dz, w2, n, H, dH, gw2, gb2, gb1); break;
    }
}

// out[c] = column sums of d [rows][C] (overwritten), C a multiple of 16 bytes
// worth of columns; part: kColBlocks * 512 floats.  Rows wider than 512 columns
// go in pieces of at most 512.
template <typename T>
static void launch_colsum(const T *d, int64_t rows, int C, float *part, float *out, cudaStream_t s) {
    for (int c0 = 0; c0 < C; c0 += 512) {
        const int w = std::min(512, C - c0), rpb = 256 / (w / (16 / (int)sizeof(T)));
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((rows + rpb - 1) / rpb, kColBlocks));
        colsum_part_kernel<T><<<g, 256, 0, s>>>(d + c0, rows, w, C, part);
        colsum_final_kernel<<<(w + 31) / 32, 256, 0, s>>>(part, g, w, out + c0);
    }
}

// Backward from t.dz through the saved activations; gradients (GEMM layout) in t.g*.
static void train_backward_enqueue(simnet_ctx *c, cudaStream_t s) {
    TrainState &t = c->tr;
    const int n = t.n_last, H = c->cfg.fc_hidden, L = c->n_layers, NO = c->n_out;
    for (int l = 0; l < L; l++) {
        if (!train_on_tc(c)) cudaMemsetAsync(t.gW[l], 0, (size_t)c->layer[l].N * c->layer[l].K * 4, s);
        cudaMemsetAsync(t.gb[l], 0, (size_t)c->layer[l].N * 4, s);
    }
    cudaMemsetAsync(t.gw2, 0, (size_t)NO * H * 4, s);
    cudaMemsetAsync(t.gb2, 0, (size_t)NO * 4, s);
    const float *Hh = t.Y[L - 1];
    if (train_on_tc(c)) {   // (the weight-gradient GEMMs overwrite gW)
        // FC2 and FC1's ReLU on the CUDA cores (2 or 22 outputs), then per layer, last
        // to first: dW = dY^T A and dA = (dY W) * [A > 0] on the tensor cores
        launch_head_bwd(Hh, t.dz, c->w2, n, H, NO, t.dHb, t.gw2, t.gb2, t.gb[L - 1], s);
        for (int l = L - 1; l >= 0; l--) {
            launch_tg(t.wgrad[l], c->cfg.spin_limit_ns, c->status, s);
            if (l < L - 1) launch_colsum(t.dYb[l & 1], layer_rows(c, l, n), c->layer[l].N, t.colpart, t.gb[l], s);
            if (l > 0) launch_tg(t.dgrad[l], c->cfg.spin_limit_ns, c->status, s);
        }
        return;
    }
    // FC2: dW2 = dz^T H, db2 = sum dz, dH = dz W2 (masked by ReLU of FC1)
    gemm(false, t.dz, 1, NO, Hh, H, 1, t.gw2, H, NO, H, n, nullptr, 0, true, s);
    colsum_kernel<<<dim3(64, 1), 32, 0, s>>>(t.dz, n, NO, t.gb2);
    float *d = t.dA, *d2 = t.dB;
    gemm(false, t.dz, NO, 1, c->w2, H, 1, d, H, n, H, NO, nullptr, 0, false, s);
    relu_mask_kernel<<<blocks((int64_t)n * H), 256, 0, s>>>(d, Hh, (int64_t)n * H);
    // FC1 and the conv layers, last to first: dW = dY^T A, db = sum dY, dA = dY W
    for (int l = L - 1; l >= 0; l--) {
        const GemmLayer &g = c->layer[l];
        const int R = (int)layer_rows(c, l, n);
        const float *A = l == 0 ? t.X : t.Y[l - 1];
        gemm(false, d, 1, g.N, A, g.K, 1, t.gW[l], g.K, g.N, g.K, R, nullptr, 0, true, s);
        launch_colsum(d, R, g.N, t.colpart, t.gb[l], s);
        if (l > 0) {
            gemm(false, d, g.N, 1, c->W32[l], g.K, 1, d2, g.K, R, g.K, g.N, nullptr, 0, false, s);
            const int64_t e = layer_rows(c, l - 1, n) * c->layer[l - 1].N;
            relu_mask_kernel<<<blocks(e), 256, 0, s>>>(d2, t.Y[l - 1], e);
            std::swap(d, d2);
        }
    }
}

// GEMM-layout gradients -> canonical blob layout (device).
static void grads_to_canonical(simnet_ctx *c, float *out, cudaStream_t s) {
    TrainState &t = c->tr;
    const simnet_config &k = c->cfg;
    const int C = k.conv_channels, H = k.fc_hidden, Ln = c->rows_n;
    float *p = out;
    int cin = kNF;
    for (int l = 0; l < k.n_conv; l++) {
        const int cin_pad = l == 0 ? kNFP : C;
        const int64_t cnt = (int64_t)C * cin * 2;
        relayout_kernel<<<blocks(cnt), 256, 0, s>>>(t.gW[l], p, 1, C, cin, 2, cin_pad, 0);
        p += cnt;
        cudaMemcpyAsync(p, t.gb[l], (size_t)C * 4, cudaMemcpyDeviceToDevice, s);
        p += C;
        cin = C;
    }
    const int64_t cnt = (int64_t)H * C * Ln;
    relayout_kernel<<<blocks(cnt), 256, 0, s>>>(t.gW[k.n_conv], p, 0, H, C, Ln, 0, 0);
    p += cnt;
    cudaMemcpyAsync(p, t.gb[k.n_conv], (size_t)H * 4, cudaMemcpyDeviceToDevice, s);
    p += H;
    cudaMemcpyAsync(p, t.gw2, (size_t)c->n_out * H * 4, cudaMemcpyDeviceToDevice, s);
    p += (size_t)c->n_out * H;
    cudaMemcpyAsync(p, t.gb2, (size_t)c->n_out * 4, cudaMemcpyDeviceToDevice, s);
}

static void refresh_shadow(simnet_ctx *c, cudaStream_t s) {
    if (c->cfg.precision != SIMNET_BF16) return;
    for (int l = 0; l < c->n_layers; l++) {
        const int64_t e = (int64_t)c->layer[l].N * c->layer[l].K;
        to_bf16_kernel<<<blocks(e), 256, 0, s>>>(c->W32[l], (__nv_bfloat16 *)c->Wl[l], e);
    }
}

// One Adam step (beta 0.9 / 0.999, eps 1e-8, no weight decay) on every parameter,
// in one launch; a BF16 context's BF16 weight copies are rewritten by it.
static void adam_all(simnet_ctx *c, float lr, cudaStream_t s) {
    TrainState &t = c->tr;
    t.step++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t.step), c2 = 1.f - powf(b2, (float)t.step);
    const bool bf16 = c->cfg.precision == SIMNET_BF16;
    AdamTable T;
    memset(&T, 0, sizeof T);
    int k = 0;
    int64_t at = 0;
    auto add = [&](float *th, float *m, float *v, const float *g, __nv_bfloat16 *sh, int64_t n) {
        T.seg[k] = AdamSeg{th, m, v, g, sh};
        T.start[k] = at;
        at += n;
        k++;
    };
    for (int l = 0; l < c->n_layers; l++) {
        const int64_t e = (int64_t)c->layer[l].N * c->layer[l].K;
        add(c->W32[l], t.mW[l], t.vW[l], t.gW[l], bf16 ? (__nv_bfloat16 *)c->Wl[l] : nullptr, e);
        add(c->bias[l], t.mb[l], t.vb[l], t.gb[l], nullptr, c->layer[l].N);
    }
    add(c->w2, t.mw2, t.vw2, t.gw2, nullptr, (int64_t)c->n_out * c->cfg.fc_hidden);
    add(c->b2, t.mb2, t.vb2, t.gb2, nullptr, c->n_out);
    T.nseg = k;
    T.start[k] = at;
    const unsigned g = (unsigned)std::min<int64_t>((at + 255) / 256, 8 * 148);
    adam_multi_kernel<<<g, 256, 0, s>>>(T, lr, b1, b2, eps, c1, c2);
}

static void invalidate_plans(simnet_ctx *c) {
    for (auto &g : c->gexec)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    c->g_B = -1;
}

extern "C" simnet_status simnet_gather_windows(simnet_ctx *c, const simnet_windows *w, const int64_t *idx, int32_t n,
                                               float *x_out, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!w || !idx || !x_out || n < 0 || !w->records || !w->fetch || !w->e_label || !w->ctx_begin)
        return fail(c, SIMNET_EINVAL, "gather_windows: bad arguments");
    if (n == 0) return SIMNET_OK;
    CK(cudaSetDevice(c->device));
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "gather_windows: no weights loaded");
    simnet_status st = ensure_train(c, n);
    if (st != SIMNET_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (train_on_tc(c))
        window_gather_kernel<__nv_bfloat16><<<blocks((int64_t)n * c->cfg.window * 16), 256, 0, s>>>(
            w->records, w->fetch, w->e_label, w->ctx_begin, idx, n, c->cfg.window, c->tr.Xb, x_out);
    else
        window_gather_kernel<float><<<blocks((int64_t)n * c->cfg.window * 16), 256, 0, s>>>(
            w->records, w->fetch, w->e_label, w->ctx_begin, idx, n, c->cfg.window, c->tr.X, x_out);
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_train_forward(simnet_ctx *c, const float *x, float *z, int32_t n, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!x || !z || n <= 0) return fail(c, SIMNET_EINVAL, "train_forward: bad arguments");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "train_forward: no weights loaded");
    if (!train_precision_ok(c)) return fail(c, SIMNET_EUNSUPPORTED, "training needs an FP32 or BF16 context of plain conv layers");
    CK(cudaSetDevice(c->device));
    simnet_status st = ensure_train(c, n);
    if (st != SIMNET_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (train_on_tc(c)) launch_pack_x<__nv_bfloat16>(x, c->tr.Xb, (int64_t)n * c->cfg.window, s);
    else launch_pack_x<float>(x, c->tr.X, (int64_t)n * c->cfg.window, s);
    st = train_forward_enqueue(c, n, s);
    if (st != SIMNET_OK) return st;
    CK(cudaMemcpyAsync(z, c->tr.z, (size_t)n * c->n_out * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_train_backward(simnet_ctx *c, const float *dz, float *grad, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!dz || !grad) return fail(c, SIMNET_EINVAL, "train_backward: bad arguments");
    if (!c->tr.ready || c->tr.n_last <= 0) return fail(c, SIMNET_ESTATE, "train_backward: no forward to differentiate");
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(c->tr.dz, dz, (size_t)c->tr.n_last * c->n_out * 4, cudaMemcpyDeviceToDevice, s));
    train_backward_enqueue(c, s);
    grads_to_canonical(c, grad, s);
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_train_loss(simnet_ctx *c, const float *z, const uint8_t *labels, int32_t n,
                                           const float *grad_scale, float *loss, float *dz, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!z || !labels || n <= 0 || (!loss && !dz)) return fail(c, SIMNET_EINVAL, "train_loss: bad arguments");
    if (c->store_queue)
        return fail(c, SIMNET_EUNSUPPORTED, "train_loss: the latency labels carry no store latency");
    CK(cudaSetDevice(c->device));
    simnet_status st = ensure_train(c, 0);   // the loss accumulator
    if (st != SIMNET_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *acc = c->tr.loss;
    CK(cudaMemsetAsync(acc, 0, sizeof(double), s));
    if (c->hybrid)
        hybrid_loss_kernel<<<blocks(2 * (int64_t)n), 256, 0, s>>>(z, labels, nullptr, n, dz, acc, grad_scale);
    else
        mse_softplus_kernel<<<blocks(2 * (int64_t)n), 256, 0, s>>>(z, labels, nullptr, n, dz, acc, grad_scale);
    if (loss) loss_to_float_kernel<<<1, 1, 0, s>>>(acc, loss);
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_train_step(simnet_ctx *c, const simnet_windows *w, const int64_t *idx, int32_t batch,
                                           float lr, float *loss_out, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!w || !idx || batch <= 0 || !w->labels || !(lr >= 0.f))
        return fail(c, SIMNET_EINVAL, "train_step: bad arguments");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "train_step: no weights loaded");
    if (!train_precision_ok(c)) return fail(c, SIMNET_EUNSUPPORTED, "training needs an FP32 or BF16 context of plain conv layers");
    if (c->store_queue)
        return fail(c, SIMNET_EUNSUPPORTED, "train_step: the training windows carry no store latency labels");
    CK(cudaSetDevice(c->device));
    simnet_status st = ensure_train(c, batch);
    if (st != SIMNET_OK) return st;
    TrainState &t = c->tr;
    cudaStream_t s = (cudaStream_t)stream;
    if (train_on_tc(c))
        window_rows_kernel<__nv_bfloat16><<<blocks((int64_t)batch * c->cfg.window, 128), 128, 0, s>>>(
            w->records, w->fetch, w->e_label, w->ctx_begin, idx, batch, c->cfg.window, t.Xb);
    else
        window_rows_kernel<float><<<blocks((int64_t)batch * c->cfg.window, 128), 128, 0, s>>>(
            w->records, w->fetch, w->e_label, w->ctx_begin, idx, batch, c->cfg.window, t.X);
    st = train_forward_enqueue(c, batch, s);
    if (st != SIMNET_OK) return st;
    CK(cudaMemsetAsync(t.loss, 0, sizeof(double), s));
    if (c->hybrid)
        hybrid_loss_kernel<<<blocks(2 * (int64_t)batch), 256, 0, s>>>(t.z, w->labels, idx, batch, t.dz, t.loss,
                                                                      nullptr);
    else
        mse_softplus_kernel<<<blocks(2 * (int64_t)batch), 256, 0, s>>>(t.z, w->labels, idx, batch, t.dz, t.loss,
                                                                       nullptr);
    train_backward_enqueue(c, s);
    adam_all(c, lr, s);
    invalidate_plans(c);
    c->weights_fp_dirty = true;
    c->const_stale = true;
    if (loss_out) {
        double l = 0.0;
        CK(cudaMemcpyAsync(&l, t.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *loss_out = (float)l;
    }
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_set_weights_device(simnet_ctx *c, const float *blob, void *stream) {
    if (!c) return SIMNET_EINVAL;
    if (!blob) return fail(c, SIMNET_EINVAL, "set_weights_device: blob is NULL");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "set_weights_device: load weights once first");
    if (!train_precision_ok(c)) return fail(c, SIMNET_EUNSUPPORTED, "needs an FP32 or BF16 context of plain conv layers");
    CK(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const simnet_config &k = c->cfg;
    const int C = k.conv_channels, H = k.fc_hidden, Ln = c->rows_n;
    const float *p = blob;
    int cin = kNF;
    for (int l = 0; l < k.n_conv; l++) {
        const int cin_pad = l == 0 ? kNFP : C;
        const int64_t cnt = (int64_t)C * cin * 2;
        relayout_kernel<<<blocks(cnt), 256, 0, s>>>(p, c->W32[l], 1, C, cin, 2, cin_pad, 1);
        p += cnt;
        CK(cudaMemcpyAsync(c->bias[l], p, (size_t)C * 4, cudaMemcpyDeviceToDevice, s));
        p += C;
        cin = C;
    }
    const int64_t cnt = (int64_t)H * C * Ln;
    relayout_kernel<<<blocks(cnt), 256, 0, s>>>(p, c->W32[k.n_conv], 0, H, C, Ln, 0, 1);
    p += cnt;
    CK(cudaMemcpyAsync(c->bias[k.n_conv], p, (size_t)H * 4, cudaMemcpyDeviceToDevice, s));
    p += H;
    CK(cudaMemcpyAsync(c->w2, p, (size_t)c->n_out * H * 4, cudaMemcpyDeviceToDevice, s));
    p += (size_t)c->n_out * H;
    CK(cudaMemcpyAsync(c->b2, p, (size_t)c->n_out * 4, cudaMemcpyDeviceToDevice, s));
    refresh_shadow(c, s);
    invalidate_plans(c);
    c->weights_fp_dirty = true;
    c->const_stale = true;
    CK(cudaGetLastError());
    return SIMNET_OK;
}

extern "C" simnet_status simnet_get_weights(simnet_ctx *c, float *blob) {
    if (!c) return SIMNET_EINVAL;
    if (!blob) return fail(c, SIMNET_EINVAL, "get_weights: blob is NULL");
    if (!c->has_weights) return fail(c, SIMNET_ESTATE, "get_weights: no weights loaded");
    if (c->residual) {   // weights only change by load_weights: the loaded blob
        memcpy(blob, c->blob_host.data(), c->blob_host.size() * sizeof(float));
        return SIMNET_OK;
    }
    CK(cudaSetDevice(c->device));
    const simnet_config &k = c->cfg;
    const int C = k.conv_channels, H = k.fc_hidden, Ln = c->rows_n;
    float *dev = nullptr;
    CK(cudaMalloc(&dev, (size_t)c->n_weights * 4));
    float *p = dev;
    int cin = kNF;
    for (int l = 0; l < k.n_conv; l++) {
        const int cin_pad = l == 0 ? kNFP : C;
        const int64_t cnt = (int64_t)C * cin * 2;
        relayout_kernel<<<blocks(cnt), 256>>>(c->W32[l], p, 1, C, cin, 2, cin_pad, 0);
        p += cnt;
        cudaMemcpy(p, c->bias[l], (size_t)C * 4, cudaMemcpyDeviceToDevice);
        p += C;
        cin = C;
    }
    const int64_t cnt = (int64_t)H * C * Ln;
    relayout_kernel<<<blocks(cnt), 256>>>(c->W32[k.n_conv], p, 0, H, C, Ln, 0, 0);
    p += cnt;
    cudaMemcpy(p, c->bias[k.n_conv], (size_t)H * 4, cudaMemcpyDeviceToDevice);
    p += H;
    cudaMemcpy(p, c->w2, (size_t)c->n_out * H * 4, cudaMemcpyDeviceToDevice);
    p += (size_t)c->n_out * H;
    cudaMemcpy(p, c->b2, (size_t)c->n_out * 4, cudaMemcpyDeviceToDevice);
    cudaError_t e = cudaMemcpy(blob, dev, (size_t)c->n_weights * 4, cudaMemcpyDeviceToHost);
    cudaFree(dev);
    if (e != cudaSuccess) return fail(c, SIMNET_ECUDA, "get_weights: %s", cudaGetErrorString(e));
    return SIMNET_OK;
}
