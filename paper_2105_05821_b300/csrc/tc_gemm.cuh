// tc_gemm.cuh -- tcgen05 tensor-core GEMM for the CNN layers (host interface).
#pragma once
#include <cuda.h>

#include <string>

#include "common.cuh"

namespace simnet {

// Everything one layer's tensor-core launch needs; built once per
// (buffers, batch capacity) and reused by every step.
struct TcPlan {
    bool ready = false;
    int prec = 0;           // SIMNET_BF16 or SIMNET_FP8_E4M3
    int BN = 0, stages = 0, grid = 0;
    int m_cap = 0, K = 0, N = 0;
    bool out_f32 = false;
    const void *in = nullptr;
    void *out = nullptr;
    size_t smem = 0;
    int64_t spin_ns = 0;
    int32_t *status = nullptr;
    CUtensorMap tA, tB;
};

// Choose tile shape and encode the TMA descriptors.  Returns false (and a
// reason) for shapes this kernel does not handle.
bool make_tc_plan(TcPlan &p, int prec, const void *in, const GemmLayer &g, void *out, bool out_f32, int m_cap,
                  int64_t spin_ns, int32_t *status, std::string &why);

// Force a tile width / stage count (the autotuner's knob); re-encodes B's map.
bool retune_tc_plan(TcPlan &p, const GemmLayer &g, int BN, int stages, std::string &why);

// C = act(A * B^T * scale + bias) * oscale for M = min(*count * m_mult, m_cap) rows.
void launch_tc_gemm(const TcPlan &p, const void *in, const GemmLayer &g, void *out, bool out_f32,
                    const int32_t *count, int m_cap, cudaStream_t s);

int num_sms();

}  // namespace simnet
