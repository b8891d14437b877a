/*
 * simnet.h -- C ABI of libsimnet, a B300 (sm_103a) implementation of SimNet's
 * data-parallel simulation loop (Li et al., "SimNet: Accurate and
 * High-Performance Computer Architecture Simulation using Deep Learning",
 * arXiv 2105.05821).
 *
 * The library simulates many independent sub-traces in lock step (Sec. 3.3).
 * Every step, for every sub-trace that still has instructions:
 *   1. gather the current instruction and its context instructions (the
 *      processor queue, newest first) into a W x 50 feature matrix (Sec. 2.2);
 *   2. run the CNN latency predictor on the whole batch (Sec. 2.3): k=2,
 *      stride-2 convolutions with ReLU, flatten, FC + ReLU, FC to the fetch
 *      and execution latencies, softplus, clamp to [0, 255], round half to
 *      even;
 *   3. advance the sub-trace's curTick by the fetch latency, retire ready
 *      queue entries in order within the retire bandwidth, evict the oldest
 *      entry of a full queue, append the instruction (Sec. 3.2);
 * and after a sub-trace's last instruction, advance its clock until the queue
 * is empty, so that its cycle count is sum(F) + Delta (Sec. 3.1, Eq. 1).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device addresses on the current device; host
 *     pointers are ordinary process memory.  Each argument says which.
 *   - The caller owns every buffer it passes.  The context owns its weights,
 *     workspaces, CUDA graphs and device status word.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; a call returns before the GPU has
 *     finished unless it fills a host output (stats, loss), in which case it
 *     synchronises the stream first.
 *   - Every call returns a simnet_status; no C++ exception crosses the ABI.
 *     On failure simnet_last_error() describes the cause.  A device-side wait
 *     that exceeds its bound makes the call return SIMNET_ETIMEOUT.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef SIMNET_H
#define SIMNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIMNET_ABI_VERSION 4
#define SIMNET_N_FEATURES 50 /* features per instruction row (Sec. 2.2) */

typedef struct simnet_ctx simnet_ctx;

typedef enum {
    SIMNET_OK = 0,
    SIMNET_EINVAL = 1,      /* bad argument: null pointer, size out of range, bad config */
    SIMNET_ENOMEM = 2,      /* device or pinned host allocation failed */
    SIMNET_ECUDA = 3,       /* a CUDA runtime/driver call failed */
    SIMNET_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    SIMNET_ESTATE = 5,      /* call out of order (e.g. simulate before load_weights) */
    SIMNET_EUNSUPPORTED = 6 /* shape/precision this build does not handle */
} simnet_status;

/* Arithmetic of the CNN.  All of them accumulate in FP32; the integer clock and
 * queue work is exact in every mode. */
typedef enum {
    SIMNET_FP32 = 0,     /* CUDA-core FFMA GEMMs */
    SIMNET_BF16 = 1,     /* tcgen05 tensor-core GEMMs, BF16 operands */
    SIMNET_FP8_E4M3 = 2  /* tcgen05 tensor-core GEMMs, FP8 e4m3 operands, per-channel scales */
} simnet_precision;

/* simnet_config.flags */
#define SIMNET_FLAG_RETIRE_STRICT 0x1u /* an entry is ready when residence > E (default: >=) */
#define SIMNET_FLAG_NO_GRAPH 0x2u      /* launch each step's kernels directly, no CUDA graph */
#define SIMNET_FLAG_KERNEL_EVENTS 0x4u /* direct launches with a CUDA event pair around each kernel;
                                          per-kernel device times via simnet_kernel_times() */
#define SIMNET_FLAG_NO_PDL 0x8u        /* no programmatic dependent launch between a step's kernels */
#define SIMNET_FLAG_LAYERWISE 0x10u    /* BF16/FP8: one kernel per layer and step (CUDA graphs,
                                          PDL, dense padding rows) instead of the default single
                                          persistent kernel that skips the padding */
#define SIMNET_FLAG_NO_CLUSTER 0x20u   /* BF16/FP8: the grid-wide persistent kernel even where the
                                          cluster kernel (SIMNET_PATH_CLUSTER) applies */
#define SIMNET_FLAG_HYBRID_HEAD 0x40u  /* hybrid latency head (Sec. 2.3): FC2 has 22 outputs, for
                                          each latency t (0 fetch, 1 execution) ten class logits
                                          z[11t+0..11t+9] and a regression output z[11t+10].  The
                                          latency is the class with the largest logit (compared in
                                          FP32, lowest index on ties) for classes 0..8, and
                                          round(clamp(softplus(z[11t+10]), 0, 255)) for class 9
                                          ("more than 8").  Without it FC2 has 2 outputs and
                                          latency t is round(clamp(softplus(z[t]), 0, 255)). */
#define SIMNET_FLAG_STORE_QUEUE 0x80u  /* store latency and memory write queue (Sec. 3.2): a third
                                          latency S per instruction (FC2 outputs 3, or 33 with the
                                          hybrid head, latency order F, E, S).  A store that retires
                                          from the processor queue enters the write queue, which
                                          retires in order, with no bandwidth limit, once a
                                          residence reaches S.  The context is every instruction in
                                          the simulator, newest first (processor queue, then write
                                          queue), at most window-1; appending to a full simulator
                                          evicts the oldest (the write queue's head first).  Context
                                          rows of stores carry S/64 in feature 44.  lat_log,
                                          pre_log and lat_replay hold 3 values per instruction. */
#define SIMNET_FLAG_RESIDUAL 0x100u    /* the n_conv layers are residual blocks (the RB models of
                                          Sec. 2.3): block k computes a = ReLU(conv(x)) and
                                          y = ReLU(pw(a) + proj(x)), conv and proj k=2 / stride-2
                                          convolutions (proj without bias), pw a pointwise
                                          convolution with bias.  Blob per block: conv.weight
                                          [C][C_in][2], conv.bias [C], pw.weight [C][C][1],
                                          pw.bias [C], proj.weight [C][C_in][2].  FP32 or BF16
                                          only (EUNSUPPORTED for FP8); runs as per-layer kernels;
                                          no device training (train_* and set_weights_device
                                          return EUNSUPPORTED) and no cnn_forward_noalloc. */
#define SIMNET_FLAG_FIXED_PATH 0x200u  /* run a whole simulate call on the path the other flags
                                          select.  Without it a long untimed BF16/FP8 call picks its
                                          path as it goes: the cluster kernel measures its padding
                                          extent over its first 128 steps and hands a batch whose
                                          queues stay long to the grid-wide kernels, and the grid-wide
                                          choice times the persistent kernel (launches of 16 and 48
                                          steps: the difference is its cost per step) and 32 steps of
                                          the per-layer kernels from the same state and runs the
                                          rest on the cheaper; the context keeps that pick for later
                                          calls with the same batch size, compaction and weights.
                                          Paths differ only in FP32 summation order;
                                          simulate_stats.path reports the last one used. */
#define SIMNET_FLAG_NO_FUSE 0x400u     /* BF16/FP8 persistent kernel: run the first two conv layers
                                          as two phases (conv1's output through device memory).
                                          By default a plain CNN of 256 channels runs them as one
                                          phase whose conv1 output stays in tensor memory as
                                          conv2's operand; both give the same values. */

/*
 * Model and simulator shape.  The CNN sees `window` rows: the current
 * instruction and up to window-1 context instructions, so the processor queue
 * holds at most window-1 entries.  `window` must be divisible by 2^n_conv.
 * Limits of this build: 2 <= window <= 256 (window-1 <= 255 queue entries),
 * 1 <= n_conv <= 8, conv_channels in {64, 128, 256}, fc_hidden a multiple of
 * 64 up to 2048, 1 <= retire_width <= 255.
 */
typedef struct {
    int32_t window;        /* W: rows given to the CNN */
    int32_t n_conv;        /* number of k=2, stride-2 conv layers */
    int32_t conv_channels; /* output channels of every conv layer */
    int32_t fc_hidden;     /* width of the first FC layer */
    int32_t retire_width;  /* processor-queue retire bandwidth, entries per cycle */
    int32_t precision;     /* simnet_precision */
    uint32_t flags;        /* SIMNET_FLAG_* */
    int32_t barrier_limit_us; /* bound on the persistent kernel's grid-barrier waits (microseconds);
                                 <= 0 uses spin_limit_ns.  When a barrier wait gives up, every CTA
                                 leaves at its next barrier (no copy in flight there) and the call
                                 returns SIMNET_ETIMEOUT; the context stays usable */
    int64_t spin_limit_ns; /* bound on any device-side wait; <= 0 selects 2 s */
} simnet_config;

/*
 * A trace already resident on the device.  Instruction record, one uint32 per
 * instruction: bits 0-4 opcode class, 5-9 src0, 10-14 src1, 15-19 dst,
 * 20 is_load, 21 is_store, 22 is_branch, 23-24 cache level (0 L1, 1 L2,
 * 2 memory), 25 mispredict; bits 26-31 must be zero.  Sub-trace b is
 * records[offsets[b] .. offsets[b+1]); offsets must be non-decreasing with
 * offsets[0] = 0 and offsets[n_subtraces] = n_instructions.  A sub-trace may
 * be empty (0 cycles) and may hold at most 4,194,303 instructions.
 */
typedef struct {
    const uint32_t *records; /* device [n_instructions] */
    const int64_t *offsets;  /* device [n_subtraces + 1] */
    int32_t n_subtraces;
    int32_t reserved;
    int64_t n_instructions;
} simnet_trace;

typedef struct {
    int64_t total_cycles; /* sum over sub-traces of their final curTick (Sec. 3.3) */
    int64_t instructions; /* instructions simulated */
    int64_t steps;        /* lock-step iterations run */
    int64_t evictions;    /* queue entries dropped at capacity */
    int64_t kernel_launches; /* kernels the call launched (graph replays counted per kernel) */
    float ms_total;          /* device time of the call, CUDA events */
    int32_t pending;         /* sub-traces not yet finished (0 once the trace is done) */
    int64_t steps_done;      /* lock-steps run since the state was initialised */
} simnet_stats;

/* Kernel kinds reported by simnet_kernel_times(). */
#define SIMNET_KERNEL_GATHER 0          /* context gather (first step, after compaction; other steps'
                                           rows come from HEAD_UPDATE) */
#define SIMNET_KERNEL_LAYER0 1          /* GEMM of layer l is SIMNET_KERNEL_LAYER0 + l (conv..., FC1) */
#define SIMNET_KERNEL_KINDS 12          /* GATHER, up to 9 GEMM layers, HEAD_UPDATE, COMPACT */
#define SIMNET_KERNEL_HEAD_UPDATE 10    /* FC2 head + clock/queue update (+ drain) + next gather */
#define SIMNET_KERNEL_COMPACT 11        /* active-set compaction */

/*
 * Autotuner: for batches of n_subtraces sub-traces, time the launch shapes of
 * the kernel path such a call takes, on a synthetic trace of `steps`
 * instructions per sub-trace, one knob after another, keeping the fastest
 * whole simnet_simulate call (the faster of two timed calls per candidate):
 *   cluster kernel:     cluster size (4 or 8 CTAs), weight-stage size (16 or
 *                       32 KB), number of weight stages (2 up to what fits);
 *   persistent kernel:  tile width (64, 128, 256 output columns) of every
 *                       tensor-core GEMM phase, then its pipeline stages (2-6);
 *   per-layer kernels:  the tile width of every tensor-core GEMM.
 * Later calls with the same batch size use the choice (simnet_autotune_plan
 * reports it).  Launch shapes change no per-element arithmetic except the
 * split of FC1's FC2 partial sums (cluster size, FC1 tile width), which moves
 * FP32 rounding only.  bn_out (host, one entry per GEMM: n_conv + 1, or
 * 3 * n_conv + 1 with SIMNET_FLAG_RESIDUAL; 25 always suffice) or NULL receives
 * the tile widths.  FP32 contexts have nothing to tune (returns OK).
 * Synchronises.  Errors: EINVAL, ESTATE (no weights), ENOMEM.
 */
simnet_status simnet_autotune(simnet_ctx *ctx, int32_t n_subtraces, int32_t steps, int32_t *bn_out,
                              void *stream);

/*
 * The last autotuner choice, into out (host, n >= 6 entries): out[0] the batch
 * size it applies to (-1: none), out[1] the kernel path it was tuned on
 * (SIMNET_PATH_*), out[2] cluster size, out[3] weight-stage bytes, out[4] weight
 * stages (cluster kernel; 0 when not tuned), out[5] pipeline stages of the
 * persistent kernel (6: as many as fit), out[6 + l] the tile width of GEMM l.
 * Errors: EINVAL (NULL pointers or n < 6).
 */
simnet_status simnet_autotune_plan(const simnet_ctx *ctx, int32_t *out, int32_t n);

/* ABI version of the loaded library (SIMNET_ABI_VERSION of its build). */
int32_t simnet_abi_version(void);

/*
 * Create a context on the current CUDA device.  `cfg` (host) is copied.
 * Allocates nothing on the device until weights or a trace arrive.
 * Errors: EINVAL for a config outside the limits above, ECUDA without a device.
 */
simnet_status simnet_init(const simnet_config *cfg, simnet_ctx **out);

/* Release every resource of the context; NULL is ignored. */
void simnet_destroy(simnet_ctx *ctx);

/* Text of the last error raised on this context (never NULL; "" if none). */
const char *simnet_last_error(const simnet_ctx *ctx);

/* Number of FP32 values in the canonical weight blob of this config. */
int64_t simnet_weight_count(const simnet_ctx *ctx);

/*
 * Load the CNN weights (Sec. 2.3).  `blob` is a HOST array of `n_values`
 * float32 in canonical order and PyTorch shapes: for k = 1..n_conv
 * conv_k.weight [C, C_in, 2] (C_in = 50 for k = 1, else C), conv_k.bias [C];
 * then fc1.weight [H, C * (W >> n_conv)] whose input index is
 * channel * (W >> n_conv) + row; fc1.bias [H]; fc2.weight [n_out, H];
 * fc2.bias [n_out].  n_out = 2 (output 0 = fetch latency, 1 = execution
 * latency), or 22 with SIMNET_FLAG_HYBRID_HEAD (outputs 11t..11t+10 for
 * latency t, in the order given there).  The library copies,
 * re-lays out and converts it to the context's precision; for FP8 it also
 * derives per-channel weight scales and, from a calibration pass over
 * synthetic context rows, per-channel activation scales.
 * Errors: EINVAL if n_values != simnet_weight_count(ctx) or blob is NULL.
 */
simnet_status simnet_load_weights(simnet_ctx *ctx, const float *blob, int64_t n_values);

/*
 * Simulate every sub-trace of `trace` to completion from an empty queue and
 * curTick = 0 (Sec. 3.2-3.3).
 *   cycles_out  device int64 [n_subtraces]: final curTick of each sub-trace.
 *   lat_log     device uint8 [n_instructions][n_lat] or NULL: the integer
 *               latencies (F, E, and S with SIMNET_FLAG_STORE_QUEUE; n_lat = 2
 *               or 3) each instruction received.
 *   pre_log     device float [n_instructions][n_lat] or NULL: softplus outputs
 *               before clamping and rounding (NaN where `lat_replay` skipped
 *               nothing: always written when non-NULL).
 *   lat_replay  device uint8 [n_instructions][n_lat] or NULL: teacher forcing; the
 *               CNN still runs (and pre_log records it) but the clock and
 *               queue use these latencies.
 *   stats       host, or NULL.  When given the call synchronises `stream`.
 * Workspaces are (re)allocated on the first call with a larger batch.
 * A trace of no sub-traces returns SIMNET_OK at once (cycles_out may then be
 * NULL); a sub-trace of no instructions finishes with 0 cycles.  A sub-trace
 * may hold at most 4,194,303 instructions, which keeps its 32-bit clock
 * (at most 255 cycles an instruction, then the drain) below 2^31.
 * Errors: EINVAL (bad trace, sub-trace longer than the limit), ESTATE (no
 * weights loaded), ENOMEM, ECUDA, ETIMEOUT.
 */
simnet_status simnet_simulate(simnet_ctx *ctx, const simnet_trace *trace, int64_t *cycles_out,
                              uint8_t *lat_log, float *pre_log, const uint8_t *lat_replay,
                              simnet_stats *stats, void *stream);

/*
 * Bounded, resumable form of simnet_simulate (checkpoint / resume of the
 * lock-step loop of Sec. 3.3).  Runs at most `max_steps` lock-step iterations
 * (max_steps < 0: until every sub-trace has finished and drained).
 *   resume = 0  start from an empty queue and curTick = 0 for every sub-trace;
 *   resume = 1  continue from the state this context holds: the state left by
 *               its previous simulate call or put there by simnet_state_load.
 *               The trace must have the same sub-trace offsets (checked by a
 *               fingerprint of `offsets` and n_instructions; the records are
 *               not checked and must be the same) and the context the same
 *               weights (checked by a fingerprint of the FP32 weights).
 * cycles_out (device int64 [n_subtraces]) receives, after every call, the
 * final curTick of each finished sub-trace and 0 for the others; lat_log,
 * pre_log and lat_replay are indexed by instruction, so a resumed call writes
 * the remaining entries of the same arrays.  stats->pending counts sub-traces
 * not yet finished; stats->steps is the iterations run by this call and
 * stats->steps_done the total since the state was initialised.  A split run
 * gives results bit-identical to an unsplit one: each row of every GEMM and
 * the FC2 partial sums depend only on the row's own inputs, and the next
 * step's feature rows are a function of the saved state alone.
 * Errors: as simnet_simulate; EINVAL for max_steps == 0 with resume == 0 is
 * not raised (the call only initialises the state); ESTATE for resume without
 * a state, with another trace or other weights.
 */
simnet_status simnet_simulate_steps(simnet_ctx *ctx, const simnet_trace *trace, int64_t *cycles_out,
                                    uint8_t *lat_log, float *pre_log, const uint8_t *lat_replay,
                                    int64_t max_steps, int32_t resume, simnet_stats *stats, void *stream);

/* Kinds of state exported by simnet_state_save. */
#define SIMNET_STATE_SIM 0   /* per-sub-trace curTick, position, queue ring, eviction counts,
                                active list and finished cycle counts */
#define SIMNET_STATE_TRAIN 1 /* FP32 master weights (canonical order), Adam moments and step */

/*
 * Export the context's state of kind `kind` into a HOST buffer.  With
 * host_buf == NULL only *bytes is set, to the size needed; otherwise *bytes
 * is the buffer's capacity on entry and the bytes written on return.  The
 * format is a versioned header (magic "SIMNETS1", the config fields that
 * shape the state, the trace and weight fingerprints) followed by the raw
 * arrays in little-endian order; it loads only into a context of the same
 * window, CNN shape and retire settings.  Synchronises `stream`.
 * Errors: EINVAL (bad kind, NULL bytes, capacity too small), ESTATE (no such
 * state: no simulate call yet, or no weights), ECUDA.
 */
simnet_status simnet_state_save(simnet_ctx *ctx, int32_t kind, void *host_buf, size_t *bytes, void *stream);

/*
 * Import a state written by simnet_state_save.  SIMNET_STATE_SIM: the next
 * simnet_simulate_steps(..., resume = 1) continues it (workspaces are sized
 * for its batch).  SIMNET_STATE_TRAIN: loads the weights as
 * simnet_load_weights does, then restores the Adam moments and step count
 * (ignored by FP8 contexts, which do not train).  Synchronises `stream`.
 * Errors: EINVAL (NULL buffer, wrong magic, version, kind or size, a state of
 * another window / CNN shape / retire setting or queue capacity), ENOMEM,
 * ECUDA.  Whether the weights match a SIM state is checked when it resumes.
 */
simnet_status simnet_state_load(simnet_ctx *ctx, int32_t kind, const void *host_buf, size_t bytes,
                                void *stream);

/*
 * Run the CNN alone on feature matrices (Sec. 2.3).
 *   x  device float [n][window][50]: rows as the simulator builds them.
 *   z  device float [n][n_out]: FC2 outputs before softplus and the class decision
 *      (n_out = 2, or 22 with SIMNET_FLAG_HYBRID_HEAD).
 * Uses the context's precision (inputs are rounded to it).
 * Errors: EINVAL (n < 0 or null pointers), ESTATE (no weights).
 */
simnet_status simnet_cnn_forward(simnet_ctx *ctx, const float *x, float *z, int32_t n,
                                 void *stream);

/*
 * Per-kernel device time of the last simnet_simulate call made with
 * SIMNET_FLAG_KERNEL_EVENTS: for each kind k < n_kinds, ms_out[k] = summed
 * CUDA-event time of its launches (milliseconds) and launches_out[k] = their
 * number (host arrays of n_kinds entries, n_kinds <= SIMNET_KERNEL_KINDS).
 * For the persistent kernel (BF16/FP8 without SIMNET_FLAG_LAYERWISE) the kinds
 * are its phases, timed by CTA 0 from barrier to barrier (globaltimer), and
 * launches_out counts phases.
 * Synchronises the device.  Errors: EINVAL (bad arguments), ESTATE (no such
 * call yet).
 */
simnet_status simnet_kernel_times(simnet_ctx *ctx, float *ms_out, int64_t *launches_out, int32_t n_kinds);

/*
 * Diagnostics of the last timed persistent-kernel call: out (host, n <= 48
 * entries) receives, for GEMM layer l, out[4l + k] = summed nanoseconds from
 * the start of the layer's phase in CTA 0 to k = 0 its first operand tile
 * arriving, 1 its last MMA commit, 2 its epilogue done, 3 the grid barrier
 * passed.  When the first two conv layers run as one phase (SIMNET_FLAG_NO_FUSE
 * not set), layer 1's row times that phase and layer 0's row holds its waits:
 * 0 the MMA warp waiting for a free accumulator, 1 for an operand unit, 2 for
 * a quarter of conv2's A operand, 3 the first epilogue warp waiting for a full
 * accumulator.  For the cluster kernel (SIMNET_PATH_CLUSTER) out[k], k < 32, is
 * the summed SM clock cycles of CTA 0's phase k instead: 0 step start (extent exchange),
 * 1 feature rows, 2/4/6 waiting for conv layer 1/2/3, 3/5/7 their epilogues
 * (7 includes the exchange of the last layer's rows), 8 waiting for FC1,
 * 9 FC1 epilogue and partial sums, 10 waiting for the partial sums, 11 head
 * and queue update, 12 extent exchange; 14 steps, 15 positions computed;
 * 18 waiting for the exchanged rows before FC1, 20 + 2l / 21 + 2l issuing
 * conv layer l's MMAs / from the last issue to the layer seen done, 26 + l
 * waiting for layer l's weight panels (26 + L: FC1's).
 * Synchronises.  Errors: EINVAL, ESTATE (no such call).
 */
simnet_status simnet_phase_detail(simnet_ctx *ctx, uint64_t *out, int32_t n);

/* Kernel paths of simnet_simulate. */
#define SIMNET_PATH_NONE 0       /* no simulate call yet */
#define SIMNET_PATH_LAYERWISE 1  /* one kernel per layer and step (CUDA graphs) */
#define SIMNET_PATH_PERSISTENT 2 /* one cooperative kernel, grid-wide barriers between phases */
#define SIMNET_PATH_CLUSTER 3    /* clusters of 4 or 8 CTAs each owning 128 sub-traces for the
                                    whole call, no grid-wide synchronisation (BF16 or FP8; 2-3 plain
                                    conv layers of 64 or 128 channels; FC1 width 256 or 512;
                                    either head, or the write queue with the regression head) */

/* Path that ran the last steps of the last simnet_simulate call (SIMNET_PATH_*), or -1 for
 * a NULL context.  A BF16/FP8 call where the cluster kernel applies starts on it; if the call is
 * longer than 512 steps and steps 64-127 needed more than two passes of last-conv positions
 * per step (long queues), the rest of the call runs on the grid-wide path.  The grid-wide
 * path of a long call is the persistent kernel or the per-layer kernels, whichever a timed
 * comparison picked (SIMNET_FLAG_FIXED_PATH: always the persistent kernel). */
int32_t simnet_kernel_path(const simnet_ctx *ctx);

/* The last timed choice between the persistent kernel and the per-layer kernels (see
 * SIMNET_FLAG_FIXED_PATH): ms_out[0] = the persistent kernel's device time for *steps_out
 * steps without its once-per-launch start, ms_out[1] = the per-layer kernels' for as many steps
 * from the same state (with their gather).  The pick also counts the persistent kernel's start.
 * All zero when no comparison has run on the context.  SIMNET_EINVAL for NULL pointers. */
simnet_status simnet_path_choice(const simnet_ctx *ctx, float *ms_out, int32_t *steps_out);

/* ------------------------------------------------------------------ training (Sec. 2.4) */

/*
 * A trace labelled by a timing model, resident on the device (all arrays
 * [n_records], indexed by instruction):
 *   fetch      cycle each instruction was fetched (non-decreasing);
 *   e_label    its execution latency label, the context feature of later windows;
 *   ctx_begin  first instruction still in flight when the previous one was
 *              fetched: the window of i holds i, then i-1 ... max(ctx_begin[i],
 *              i-window+1), with residence fetch[i-1] - fetch[j];
 *   labels     [n_records][2] (fetch, execution) latency targets.
 */
typedef struct {
    const uint32_t *records;
    const int64_t *fetch;
    const uint8_t *e_label;
    const int64_t *ctx_begin;
    const uint8_t *labels;
    int64_t n_records;
} simnet_windows;

/*
 * Feature matrices of the windows idx[0..n) (device int64, each in
 * [0, n_records)) into x_out (device float [n][window][50]), the same rows the
 * simulator builds.  Errors: EINVAL, ESTATE (no weights loaded).
 */
simnet_status simnet_gather_windows(simnet_ctx *ctx, const simnet_windows *w, const int64_t *idx, int32_t n,
                                    float *x_out, void *stream);

/*
 * CNN forward for training: x device float [n][window][50], z device float
 * [n][n_out] (FC2 outputs before softplus).  Keeps every layer's output for the next
 * simnet_train_backward (one forward is kept per context).  FP32 contexts
 * compute in FP32 on the CUDA cores; BF16 contexts use autocast numerics on the
 * tcgen05 tensor cores: the windows, the conv layers' outputs and their
 * gradients are BF16, sums FP32, FC1's output, FC2 and the loss FP32.
 * Errors: EINVAL, ESTATE, EUNSUPPORTED (FP8).
 */
simnet_status simnet_train_forward(simnet_ctx *ctx, const float *x, float *z, int32_t n, void *stream);

/*
 * Backward of the last simnet_train_forward: dz device float [n][n_out] (dLoss/dz),
 * grad device float [simnet_weight_count] receives dLoss/dtheta in the
 * canonical blob layout of simnet_load_weights (overwritten).
 * Errors: EINVAL, ESTATE (no forward yet).
 */
simnet_status simnet_train_backward(simnet_ctx *ctx, const float *dz, float *grad, void *stream);

/*
 * The training loss of Sec. 2.4 on FC2 outputs, and its gradient.
 *   z           device float [n][n_out] (FC2 outputs before softplus).
 *   labels      device uint8 [n][2]: the (fetch, execution) latency labels of row r.
 *   grad_scale  device float [1] or NULL (= 1): multiplies dz (the incoming
 *               gradient of an autograd graph).
 *   loss        device float [1] or NULL: the mean over the 2n latencies of
 *               (softplus(z) - label)^2; with SIMNET_FLAG_HYBRID_HEAD plus the
 *               cross-entropy of each latency's ten class logits against class
 *               min(label, 9).
 *   dz          device float [n][n_out] or NULL: grad_scale * dloss/dz.
 * The same arithmetic as simnet_train_step's loss.  Errors: EINVAL (null z or
 * labels, n <= 0, or neither output), EUNSUPPORTED (SIMNET_FLAG_STORE_QUEUE:
 * no store-latency labels).
 */
simnet_status simnet_train_loss(simnet_ctx *ctx, const float *z, const uint8_t *labels, int32_t n,
                                const float *grad_scale, float *loss, float *dz, void *stream);

/*
 * One training step on the windows idx[0..batch) (device int64): gather, forward,
 * loss = mean over the 2*batch latencies of (softplus(z) - label)^2 (labels are
 * 0..255; z the regression output of the latency); with SIMNET_FLAG_HYBRID_HEAD
 * each latency adds the cross-entropy of its ten class logits against class
 * min(label, 9) (Sec. 2.3); backward, and an Adam step (beta 0.9/0.999, eps 1e-8, no weight
 * decay) with learning rate lr on FP32 master weights; a BF16 context's BF16
 * weights are refreshed from them.  loss_out (host) or NULL; when given the call
 * synchronises `stream`.  Later simulate/cnn_forward calls use the new weights.
 */
simnet_status simnet_train_step(simnet_ctx *ctx, const simnet_windows *w, const int64_t *idx, int32_t batch,
                                float lr, float *loss_out, void *stream);

/* Replace the weights from a DEVICE blob in canonical layout (FP32/BF16 contexts). */
simnet_status simnet_set_weights_device(simnet_ctx *ctx, const float *blob, void *stream);

/* Current weights (FP32 master copy) into a HOST blob in canonical layout.  Synchronises. */
simnet_status simnet_get_weights(simnet_ctx *ctx, float *blob);

/*
 * simnet_cnn_forward_noalloc: simnet_cnn_forward for callers that cannot
 * allocate device memory while they run (inside an allocator or memory-pool
 * callback, under a device-memory budget reserved up front by another
 * framework, or in a latency-critical loop that cannot take cudaMalloc's
 * implicit synchronisation).  The paper has no counterpart; it is a property
 * of this library's interface.
 *   x, z, n, stream  as simnet_cnn_forward (x device float [n][window][50],
 *                    z device float [n][n_out], FC2 outputs before softplus).
 * The context must use SIMNET_FP32 and have weights loaded, else
 * SIMNET_EUNSUPPORTED.  The call allocates nothing: its workspace is a
 * file-scope device array of SIMNET_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until process exit.  It needs
 *   256 + 4*n*window*64 + 2*4*n*(window/2)*conv_channels + 4*n*fc_hidden
 * bytes (each term rounded up to 256); a larger n returns SIMNET_EINVAL with
 * the sizes in simnet_last_error().  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture that should contain this entry point.  All calls
 * share the array and it keeps the previous call's contents (each call
 * overwrites every byte it reads); calls whose GPU work overlaps race on it.
 */
#define SIMNET_NOALLOC_SCRATCH_BYTES (16u << 20)
simnet_status simnet_cnn_forward_noalloc(simnet_ctx *ctx, const float *x, float *z, int32_t n,
                                         void *stream);
/* Size in bytes of the fixed scratch array behind simnet_cnn_forward_noalloc. */
size_t simnet_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* SIMNET_H */
