// train_tc.cuh -- tcgen05 GEMMs of the BF16 training step (host interface).
#pragma once
#include <cuda.h>

#include <string>

#include "common.cuh"

namespace simnet {

// What a training GEMM's epilogue does with C[m][n] = sum_r A(m, r) B(n, r).
enum TgEpi : int {
    TG_FWD_BF16 = 0,  // out bf16 [M][N] = ReLU(C + bias[n])
    TG_FWD_F32 = 1,   // out f32 [M][N] = ReLU(C + bias[n]); a split reduction writes each split's
                      // raw tile to `part` [splits][M][N], summed, biased and ReLU'd afterwards
    TG_DGRAD = 2,     // out bf16 [M][N] = C where mask[m][n] > 0, else 0 (ReLU derivative)
    TG_WGRAD = 3,     // out f32 [N][ldo]: out[n][m] = C; a reduction split over the CTAs writes
                      // each split's tile to `part` [splits][N][ldo], summed into out afterwards
};

// One training GEMM, built once per (buffers, sizes) and launched every step.
//   A(m, r): K-major, stored [M][R] (a_mn = false), or MN-major, stored [R][M] (a_mn = true)
//   B(n, r): K-major, stored [N][R] (b_mn = false), or MN-major, stored [R][N] (b_mn = true)
// All operands BF16; R is padded to a multiple of 64 by zero fill (TMA out-of-bounds reads).
struct TgPlan {
    bool ready = false;
    int epi = 0, BN = 0, stages = 0, grid = 0;
    bool a_mn = false, b_mn = false;
    int M = 0, N = 0, R = 0, ldo = 0;
    int n_tiles_n = 0, m_tiles = 0, splits = 1, kb_per_split = 0;
    size_t smem = 0;
    const float *bias = nullptr;
    const void *mask = nullptr;
    void *out = nullptr;
    float *part = nullptr;   // split reductions: the caller's scratch of tg_part_floats(p) floats
    CUtensorMap tA, tB;
};

// Floats of split scratch a TG_WGRAD plan needs (0 when it does not split).
inline size_t tg_part_floats(const TgPlan &p) {
    if (p.splits <= 1) return 0;
    if (p.epi == TG_WGRAD) return (size_t)p.splits * p.N * p.ldo;
    if (p.epi == TG_FWD_F32) return (size_t)p.splits * p.M * p.N;
    return 0;
}

// Describe C = A * B^T for the given storage; returns false (and why) for
// shapes the kernel does not take (N not a multiple of 64, or of BN).
bool make_tg_plan(TgPlan &p, int epi, const void *A, bool a_mn, const void *B, bool b_mn, int M, int N, int R,
                  void *out, int ldo, const float *bias, const void *mask, std::string &why);

void launch_tg(const TgPlan &p, int64_t spin_ns, int32_t *status, cudaStream_t s);

}  // namespace simnet
