// noalloc.cu -- simnet_cnn_forward_noalloc: the CNN-only entry point with its
// workspace in a fixed, file-scope device array instead of cudaMalloc'd memory.
//
// Who needs it: callers that must not allocate device memory while they run,
// e.g. code inside an allocator or memory-pool callback, a process whose device
// memory is reserved up front by another framework, or a latency-critical loop
// that cannot afford cudaMalloc's implicit device synchronisation.  They pass
// inputs and outputs; this call allocates nothing (no cudaMalloc, cudaFree,
// pinned host memory or library allocation).
//
// The array below is part of the library image: every GPU that loads
// libsimnet.so holds SIMNET_NOALLOC_SCRATCH_BYTES of device memory until the
// process exits.  Host code may not use the array's name as a device address
// (on the host it names a stand-in); the address comes from
// cudaGetSymbolAddress, taken once per device on the first call with that
// device current.  That first call should therefore happen before any stream
// capture that includes this entry point.  All calls share the array and it
// keeps the last call's contents; calls whose GPU work overlaps (other streams,
// other threads) race on it.  Nothing in it needs clearing: every call writes
// each byte it later reads (row count, features, activations).  The row count
// is written by a one-thread kernel that takes it by value, so no host memory
// is read while the call's work runs.  The caller's current device is restored
// before every return.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SIMNET_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void set_count_kernel(int32_t *count, int32_t n) { *count = n; }

// Makes `dev` current for the scope and puts the caller's device back after.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

using namespace simnet;

extern "C" size_t simnet_noalloc_scratch_bytes(void) { return (size_t)SIMNET_NOALLOC_SCRATCH_BYTES; }

extern "C" simnet_status simnet_cnn_forward_noalloc(simnet_ctx *c, const float *x, float *z, int32_t n,
                                                    void *stream) {
    if (!c) return SIMNET_EINVAL;
    CtxFp32View v;
    if (!ctx_fp32_view(c, v)) {
        ctx_set_error(c, "cnn_forward_noalloc: needs an FP32 context with weights loaded");
        return SIMNET_EUNSUPPORTED;
    }
    if (n < 0 || (n > 0 && (!x || !z))) {
        ctx_set_error(c, "cnn_forward_noalloc: bad arguments");
        return SIMNET_EINVAL;
    }
    // workspace: count | X [n][W][64] | act0, act1 [n][W/2][C] | h1 [n][H]   (FP32)
    const GemmLayer &g0 = v.layer[0];
    const size_t xb = round256((size_t)n * v.window * kNFP * sizeof(float));
    const size_t ab = round256((size_t)n * g0.m_mult * g0.N * sizeof(float));
    const size_t hb = round256((size_t)n * v.hidden * sizeof(float));
    const size_t need = 256 + xb + 2 * ab + hb;
    if (need > (size_t)SIMNET_NOALLOC_SCRATCH_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf, "cnn_forward_noalloc: %d windows need %zu bytes of scratch, the limit is %zu",
                 n, need, (size_t)SIMNET_NOALLOC_SCRATCH_BYTES);
        ctx_set_error(c, buf);
        return SIMNET_EINVAL;
    }
    if (n == 0) return SIMNET_OK;
    if (v.device < 0 || v.device >= kMaxDevices) {
        ctx_set_error(c, "cnn_forward_noalloc: cannot select the context's device");
        return SIMNET_ECUDA;
    }
    DeviceGuard guard(v.device);
    if (!guard.ok) {
        ctx_set_error(c, "cnn_forward_noalloc: cannot select the context's device");
        return SIMNET_ECUDA;
    }
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[v.device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                char buf[160];
                snprintf(buf, sizeof buf, "cnn_forward_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                ctx_set_error(c, buf);
                return SIMNET_ECUDA;
            }
            g_scratch_addr[v.device] = (unsigned char *)p;
        }
        base = g_scratch_addr[v.device];
    }
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *count = (int32_t *)base;
    float *X = (float *)(base + 256);
    float *act[2] = {(float *)(base + 256 + xb), (float *)(base + 256 + xb + ab)};
    float *h1 = (float *)(base + 256 + xb + 2 * ab);
    // the row count the GEMMs read, passed by value to a one-thread kernel
    set_count_kernel<<<1, 1, 0, s>>>(count, n);
    launch_pack_x<float>(x, X, (int64_t)n * v.window, s);
    const float *in = X;
    for (int l = 0; l < v.n_layers; l++) {
        const GemmLayer &g = v.layer[l];
        float *out = l == v.n_layers - 1 ? h1 : act[l & 1];
        launch_gemm_f32(in, (const float *)g.B, g.bias, out, count, g.m_mult, n * g.m_mult, g.N, g.K, g.relu, s);
        in = out;
    }
    launch_head_z(h1, v.w2, v.b2, z, n, v.hidden, v.n_out, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof buf, "cnn_forward_noalloc: launch failed: %s", cudaGetErrorString(e));
        ctx_set_error(c, buf);
        return SIMNET_ECUDA;
    }
    return SIMNET_OK;
}
