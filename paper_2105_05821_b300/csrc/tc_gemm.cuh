// tc_gemm.cuh -- tcgen05 tensor-core GEMM for the CNN layers (host interface).
#pragma once
#include <cuda.h>

#include <string>

#include "common.cuh"

namespace simnet {

// What the epilogue writes.
enum TcOut : int {
    TC_OUT_ACT = 0,   // activations [M][N] in the layer precision (BF16, or FP8 e4m3)
    TC_OUT_F32 = 1,   // FP32 [M][N]
    TC_OUT_PART = 3,  // FC2 partial dot products [2*N/BN][m_cap][2] float (fetch, execution)
    TC_OUT_PART_HYBRID = 4,  // the same for the hybrid head's 22 FC2 outputs: [2*N/BN][m_cap][22]
    TC_OUT_PART3 = 5,        // ... three regression outputs (fetch, execution, store)
    TC_OUT_PART33 = 6,       // ... the hybrid head with the store latency (33 outputs)
};

// Everything one layer's tensor-core launch needs; built once per
// (buffers, batch capacity) and reused by every step.
struct TcPlan {
    bool ready = false;
    int prec = 0;           // SIMNET_BF16 or SIMNET_FP8_E4M3
    int BN = 0, stages = 0, grid = 0;
    int m_cap = 0, K = 0, N = 0;
    int out_kind = TC_OUT_ACT;
    int prm_floats = 0;
    bool pdl = false;
    const void *in = nullptr;
    const void *wB = nullptr;
    void *out = nullptr;
    const void *resid = nullptr;   // residual block: [m_cap][N] added before the activation
    size_t smem = 0;
    int64_t spin_ns = 0;
    int32_t *status = nullptr;
    CUtensorMap tA, tB;
};

// Choose tile shape and encode the TMA descriptors.  Returns false (and a
// reason) for shapes this kernel does not handle.
bool make_tc_plan(TcPlan &p, int prec, const void *in, const GemmLayer &g, void *out, int out_kind, int m_cap,
                  int64_t spin_ns, int32_t *status, bool pdl, std::string &why, const void *resid = nullptr);

// Force a tile width (the autotuner's knob); re-encodes B's map.
bool retune_tc_plan(TcPlan &p, const GemmLayer &g, int BN, std::string &why);

// C = act(A * B^T * scale + bias) * oscale for M = min(*count * m_mult, m_cap)
// rows; TC_OUT_PART / TC_OUT_PART_HYBRID fold FC2 (`w2` [2][N] / [22][N]) into
// the epilogue instead.
void launch_tc_gemm(const TcPlan &p, const GemmLayer &g, const int32_t *count, const float *w2, cudaStream_t s);

int num_sms();

// 2D tiled TMA map (128-byte swizzle) over a row-major [outer][inner] array.
bool encode_map_2d(CUtensorMap &m, int prec, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                   uint32_t box_outer, std::string &why);

}  // namespace simnet
