"""Benchmark: simulated instructions per second of SimNet's lock-step sub-trace
simulation on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--precision bf16]
    python bench.py --impl reference ...      # the FP64 CPU oracle on the host cores

One step = one full simnet_simulate call over the workload's whole trace:
every lock-step iteration (gather, conv GEMMs, FC1, head + queue update), the
drains and the per-sub-trace cycle counts.  Inputs are resident in HBM before
the timed region; L2 is flushed (512 MB write) before every timed step and the
flush is outside the step's CUDA-event pair.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import faulthandler
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2105_05821_b300 import inputs as I  # noqa: E402

METRIC = "simulated instr/sec on 1 B300 (BF16/FP8 vs FP32 form) at stated CPI error"
UNIT = "inst/s"
FP32_FMA_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
# DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel,
# keyed by (workload, precision, kernel); from the capture summarised in profiles/.
TRAFFIC = {
    # persist_kernel, c2 BF16: 1.53 MB of DRAM traffic over 20 steps in the capture of
    # profiles/persist_kernel_c2_bf16.md, scaled by steps to the 1,000-step launch
    ("c2", "bf16", "persist_kernel"): 1.526e6 * 1000 / 20,
    # cluster_kernel, c2: one 1,000-step call is two launches (the 128-step probe and the
    # rest), measured on the full workload; nothing is written, the working set stays on
    # chip and in L2 (profiles/cluster_kernel_c2_bf16_traffic.md: mean of seven calls;
    # ..._fp8_traffic.md)
    ("c2", "bf16", "cluster_kernel"): 2.248411e6 + 5.413998e6,
    ("c2", "fp8", "cluster_kernel"): 1.872896e6 + 5.331968e6,
    # persist_kernel, c5 (conv1 and conv2 in one phase): 158.23 GB (BF16) and 74.25 GB (FP8)
    # over one call of 65,536 sub-traces cut to 100 instructions (ncu, one pass;
    # profiles/persist_kernel_c5_fused.md), scaled by instructions to the 100M-instruction
    # launch (the traffic a step follows the active sub-traces: one instruction each)
    ("c5", "bf16", "persist_kernel"): 158.22559488e9 * 1e8 / 6_553_600,
    ("c5", "fp8", "persist_kernel"): 74.252812032e9 * 1e8 / 6_553_600,
}


def traffic_of(args, workload, prec, kernel):
    """TRAFFIC's figure for a launch of the whole workload; none for a cut one."""
    return None if getattr(args, "subtrace_len", 0) else TRAFFIC.get((workload, prec, kernel))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p["bf16_tflops_sustained"], "measured"
    except Exception:
        return 6400.0, 1800.0, 1400.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle timing
def oracle_rate(w: I.Workload, trace: I.Trace, blob, ids, threads=0):
    """Instructions/s of the FP64 oracle on the listed sub-traces (host cores)."""
    import oracle
    cfg = oracle.Config.of(w.arch, retire_width=w.retire_width)
    n = int(sum(trace.offsets[i + 1] - trace.offsets[i] for i in ids))
    t0 = time.perf_counter()
    r = oracle.simulate(cfg, trace.records, trace.offsets, blob, subset=ids, n_threads=threads)
    dt = time.perf_counter() - t0
    return n / dt, n, dt, r


def host_cores():
    """CPUs this process may really use: affinity mask, capped by a cgroup CPU quota."""
    n = len(os.sched_getaffinity(0))
    try:
        q, per = open("/sys/fs/cgroup/cpu.max").read().split()[:2]
        if q != "max":
            n = min(n, max(1, int(-(-int(q) // int(per)))))
    except Exception:
        pass
    return n


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_sample_ids(w, trace, blob, target_s=15.0):
    """A bounded sample of whole sub-traces sized for ~target_s of oracle work,
    calibrated on one wave of sub-traces (one per thread)."""
    threads = host_cores()
    ids = list(range(min(threads, trace.n_subtraces)))
    rate, _, dt, _ = oracle_rate(w, trace, blob, ids, threads=threads)
    avg_len = trace.n_instructions / trace.n_subtraces
    n = int(min(trace.n_subtraces, rate * target_s / avg_len))
    n = max(len(ids), (n // threads) * threads)
    return list(range(min(n, trace.n_subtraces))), threads


def workload_of(args) -> I.Workload:
    """The named workload, with the hybrid latency head (Sec. 2.3) and the store
    latency with the memory write queue (Sec. 3.2) on request."""
    w = I.WORKLOADS[args.workload]
    head = getattr(args, "head", "regression")
    store = bool(getattr(args, "store_queue", False))
    if head != "regression" or store:
        a = w.arch
        w = dataclasses.replace(w, arch=I.Arch(a.window, a.n_conv, a.channels, a.hidden, head, store, a.block))
    return w


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload_of(args)
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    threads = host_cores()
    per_step = threads                      # one sub-trace per host thread per step
    times, insts = [], []
    for s in range(args.warmup + args.steps):
        lo = (s * per_step) % trace.n_subtraces
        ids = [(lo + j) % trace.n_subtraces for j in range(per_step)]
        rate, n, dt, _ = oracle_rate(w, trace, blob, ids, threads=threads)
        if s >= args.warmup:
            times.append(dt)
            insts.append(n)
    value = sum(insts) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, args, note="each step a sample of "
                                                          f"{per_step} whole sub-traces"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} whole sub-traces per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, args, note=""):
    c = {"workload": f"{w.name}: {w.description}; weights: {I.weight_recipe(w)}", "n_subtraces": w.n_subtraces,
         "instructions_per_step": None, "window": w.arch.window, "n_conv": w.arch.n_conv,
         "channels": w.arch.channels, "fc_hidden": w.arch.hidden, "retire_width": w.retire_width,
         "precision": args.precision, "head": w.arch.head, "store_queue": w.arch.store_queue,
         "block": w.arch.block,
         "l2": "flushed (512 MB write) before every timed step"}
    if note:
        c["note"] = note
    return c


# ----------------------------------------------------------------------------- our arm
def algorithmic_units(w: I.Workload, kind: int, n_active: float, prec: str):
    """(amount, unit, bound) per step of kernel kind `kind` for n_active
    sub-traces (a residual block's kind covers its three GEMMs)."""
    a = w.arch
    es = {"fp32": 4, "bf16": 2, "fp8": 1}[prec]
    if 1 <= kind <= a.n_conv + 1:
        l = kind - 1
        if l < a.n_conv:
            rows = a.window >> (l + 1)
            cin = I.N_FEATURES if l == 0 else a.channels
            macs = rows * a.channels * cin * 2
            if a.block == "residual":   # the block's three GEMMs: conv, projection, pointwise
                macs = 2 * rows * a.channels * cin * 2 + rows * a.channels * a.channels
        else:
            macs = a.fc1_in * a.hidden
        return 2.0 * macs * n_active, "flop", ("alu" if prec == "fp32" else "tensor")
    if kind == 0:   # gather: feature tile written, ring + record + scalars read
        per = a.window * 64 * es + (a.window - 1) * 8 + 4 + 16
        return per * n_active, "byte", "hbm"
    if kind == 10:  # head + update + next gather: FC2 partials, ring, append, scalars, next tile rows
        parts = a.hidden // 64
        per = parts * 4 * a.n_out + (a.window - 1) * 8 + 8 + 4 + 32 + a.window * 64 * es
        return per * n_active, "byte", "hbm"
    return 0.0, "byte", "hbm"


KIND_NAMES = {0: "gather", 10: "head_update", 11: "compact"}


def kind_name(w, k):
    if k in KIND_NAMES:
        return KIND_NAMES[k]
    l = k - 1
    if l < w.arch.n_conv:
        return f"rb{l + 1}_gemms" if w.arch.block == "residual" else f"conv{l + 1}_gemm"
    return "fc1_gemm"


def train_predictor(w: I.Workload, steps: int):
    """The uneven-batching workload uses a trained CNN: train its architecture
    (window 96) with the library's fused steps on toy-pipeline labels of the
    training workload's trace (batch 4096, Adam lr 1e-3)."""
    import torch
    from paper_2105_05821_b300.simnet import Simnet
    from paper_2105_05821_b300.train import Windows, train
    tw = I.WORKLOADS["c3"]
    rec = I.make_records(tw.n_instructions, tw.seed)
    win = Windows.from_labels(rec, I.toy_labels(rec))
    sim = Simnet.for_arch(w.arch, precision="fp32")
    sim.load_weights(I.workload_weights(w).astype(np.float32))
    t0 = time.perf_counter()
    losses = train(sim, win, steps, 4096, lr=1e-3, seed=w.seed)
    torch.cuda.synchronize()
    info = {"steps": steps, "batch": 4096, "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:])),
            "seconds": time.perf_counter() - t0, "labels": "toy pipeline model on the training trace (2M)"}
    blob = sim.get_weights()
    sim.close()
    return blob, info


def truncate(trace: I.Trace, n: int) -> I.Trace:
    lens = np.minimum(trace.lengths(), n)
    parts = [trace.records[trace.offsets[b]:trace.offsets[b] + lens[b]] for b in range(trace.n_subtraces)]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return I.Trace(np.concatenate(parts).astype(np.uint32), offs)


class Timer:
    """CUDA-event timing of whole simnet_simulate calls on one device: L2
    flushed (512 MB write) before every timed call, outside its event pair."""

    def __init__(self, dev):
        import torch
        self.torch = torch
        self.dev = dev
        self.flush = torch.empty(128 * 1024 * 1024, dtype=torch.int32, device=dev)   # 512 MB > L2

    def run(self, sim, rec, off, cyc, steps, warmup, e2e=None):
        """Device ms of each of `steps` calls after `warmup` untimed ones.  With
        e2e = (rec_h, off_h, cyc_h) every timed call also copies the trace from
        pinned host memory and the cycle counts back inside its event pair."""
        torch = self.torch
        for _ in range(warmup):
            sim.simulate(rec, off, cycles_out=cyc, stats=False)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            self.flush.zero_()
            evs[i][0].record()
            if e2e:
                rec.copy_(e2e[0], non_blocking=True)
                off.copy_(e2e[1], non_blocking=True)
            sim.simulate(rec, off, cycles_out=cyc, stats=False)
            if e2e:
                e2e[2].copy_(cyc, non_blocking=True)
            evs[i][1].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return [a.elapsed_time(b) for a, b in evs], wall


def tensor_peak(prec: str, call_ms: float):
    """The tensor roofline's denominator: the measured BF16 burst peak for a call
    shorter than 0.2 s (one call timed alone between L2 flushes), the sustained
    one for a longer call; FP8 takes twice the BF16 figure (nominal ratio)."""
    hbm, burst, sus, src = peaks()
    base, which = (burst, "burst") if call_ms < 200.0 else (sus, "sustained")
    scale = 2.0 if prec == "fp8" else 1.0
    return base * scale, f"{src} bf16 {which}" + (" x2 (fp8 nominal ratio)" if scale > 1 else "")


def whole_call_roofline(w, prec, N, ms_per_step, kernel, traffic=None):
    """One launch (or one kernel path) does the whole call: its algorithmic
    FLOPs (dense count of the scope table) over the call's device time."""
    flops = 2.0 * w.arch.macs_per_inference() * N
    ach = flops / (ms_per_step / 1e3) / 1e12
    peak, note = tensor_peak(prec, ms_per_step)
    return {"kernel": kernel, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "peak_source": note, "traffic": traffic, "avg_launch_us": ms_per_step * 1e3,
            "algorithmic_per_launch": flops, "algorithmic_unit": "flop", "share_of_step": 1.0}


PATH_KERNEL = {"cluster": "cluster_kernel", "persistent": "persist_kernel", "layerwise": "per-layer kernels"}


def measure(timer, w, trace, blob32, prec, steps, warmup, rec, off, autotune=False, **kw):
    """One context of workload `w` at precision `prec`: its first (untimed)
    call runs any path choice, then `steps` timed calls.  Returns the record
    and the per-sub-trace cycles of the last call."""
    import torch
    from paper_2105_05821_b300.simnet import Simnet
    N, B = trace.n_instructions, trace.n_subtraces
    cyc = torch.empty(B, dtype=torch.int64, device=rec.device)
    sim = Simnet.for_arch(w.arch, precision=prec, retire_width=w.retire_width, **kw)
    sim.load_weights(blob32)
    st = sim.simulate(rec, off, cycles_out=cyc, stats=True)
    tiles = []
    if autotune and prec != "fp32" and sim.kernel_path != "cluster":
        tiles = sim.autotune(B)
        st = sim.simulate(rec, off, cycles_out=cyc, stats=True)
    ms, wall = timer.run(sim, rec, off, cyc, steps, warmup)
    ms_per_step = sum(ms) / len(ms)
    rec_out = {"value": N / (ms_per_step / 1e3), "unit": UNIT, "ms_per_step": ms_per_step,
               "ms_range": [min(ms), max(ms)], "steps": steps, "warmup": warmup, "dtype": prec,
               "kernel_mode": sim.kernel_path, "gpu_launches_per_step": int(st.kernel_launches),
               "total_cycles": int(st.total_cycles), "cpi": st.total_cycles / N, "wall_s_timed": wall}
    if tiles:
        rec_out["tile_widths"] = tiles[:w.arch.n_conv + 1]
    pc = sim.path_choice
    if pc["steps"]:
        rec_out["path_choice"] = pc
    cycles = cyc.cpu().numpy()
    return sim, rec_out, cycles


def device_trace(trace, dev):
    import torch
    rec_h = torch.from_numpy(trace.records.view(np.int32).copy()).pin_memory()
    off_h = torch.from_numpy(trace.offsets.copy()).pin_memory()
    return rec_h, off_h, rec_h.to(dev), off_h.to(dev)


def cpi_error(gpu_cycles, ids, oracle_cycles):
    return abs(float(np.asarray(gpu_cycles)[ids].sum()) / float(np.asarray(oracle_cycles).sum()) - 1.0)


def run_ours(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    timer = Timer(dev)
    w = workload_of(args)
    trace = I.make_trace(w)
    if args.subtrace_len:
        trace = truncate(trace, args.subtrace_len)
    blob32 = I.workload_weights(w).astype(np.float32)
    train_info = None
    if args.workload == "c4" and not args.untrained and not w.arch.store_queue:   # no store labels to train on
        blob32, train_info = train_predictor(w, args.train_steps)
    N, B = trace.n_instructions, trace.n_subtraces
    rec_h, off_h, rec, off = device_trace(trace, dev)
    cyc_h = torch.empty(B, dtype=torch.int64).pin_memory()
    kw = dict(persistent=not args.layerwise, cluster=not args.no_cluster, auto_path=not args.fixed_path)

    with ClockSampler(dev.index) as clk:
        sim, main, cycles = measure(timer, w, trace, blob32, args.precision, args.steps, args.warmup, rec, off,
                                    autotune=not args.no_autotune, **kw)
    clocks = clk.summary()
    path = main["kernel_mode"]
    # end to end through host buffers (pinned H2D of the trace, D2H of the cycle counts)
    cyc = torch.empty(B, dtype=torch.int64, device=dev)
    ms_e2e, _ = timer.run(sim, rec, off, cyc, max(2, args.steps // 2), 1, e2e=(rec_h, off_h, cyc_h))
    e2e_value = N / (sum(ms_e2e) / len(ms_e2e) / 1e3)
    sim.close()

    out = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
           "config": workload_config(w, args), "clocks": clocks,
           "gpu_launches": int(main["gpu_launches_per_step"] * args.steps),
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(4 * N + 8 * (B + 1)),
                   "d2h_bytes_per_step": int(8 * B)},
           "wall_s_timed": main["wall_s_timed"], "ms_range": main["ms_range"],
           "tile_widths": main.get("tile_widths", []),
           "kernel_mode": {"layerwise": "per-layer kernels", "persistent": "persistent",
                           "cluster": "cluster"}.get(path, path)}
    if "path_choice" in main:
        out["path_choice"] = main["path_choice"]   # the timed persistent / per-layer comparison behind kernel_mode
    out["config"]["instructions_per_step"] = N
    out["total_cycles"] = main["total_cycles"]
    out["cpi"] = main["cpi"]

    if not args.no_breakdown and path == "cluster":
        # one launch does every step: the whole call's algorithmic work over its device time
        out["roofline"] = whole_call_roofline(w, args.precision, N, main["ms_per_step"], "cluster_kernel",
                                              traffic_of(args, w.name, args.precision, "cluster_kernel"))
        ph = cluster_phases(w, args, blob32, rec, off, clocks.get("sm_mhz") or 2032.0)
        out["phases_us_per_step"] = ph
        # the padding extent: the kernel computes only the last-conv positions below
        # the longest queue, so it executes a fraction of the dense FLOPs
        frac_pos = ph["positions_per_step"] / w.arch.rows_out
        exe = 2.0 * (frac_pos * (w.arch.macs_per_inference() - w.arch.n_out * w.arch.hidden)
                     + w.arch.n_out * w.arch.hidden) * N
        out["roofline"]["executed_flop"] = exe
        out["roofline"]["executed_tflops"] = exe / (main["ms_per_step"] / 1e3) / 1e12
        out["roofline"]["executed_note"] = (f"positions computed per step {ph['positions_per_step']:.2f} of "
                                            f"{w.arch.rows_out} (CTA 0's counter); conv and FC1 scale with "
                                            "them, FC2 does not")
    elif not args.no_breakdown:
        roof, kernels = roofline(w, args, blob32, rec, off, B, path)
        out["kernels"] = kernels
        out["roofline"] = roof
        if path == "persistent":
            # one launch does every step: its roofline is the whole call's work over its
            # device time; the per-phase table explains the split
            out["roofline"] = whole_call_roofline(w, args.precision, N, main["ms_per_step"], "persist_kernel",
                                                  traffic_of(args, w.name, args.precision, "persist_kernel"))
            out["roofline"]["dominant_phase"] = roof

    forms = {}
    if args.precision != "fp32" and not args.no_fp32:
        s32, r32, c32 = measure(timer, w, trace, blob32, "fp32", max(2, args.steps // 3), 1, rec, off)
        s32.close()
        r32["note"] = "FFMA CUDA-core GEMMs, per-layer kernels, same workload and timing"
        out["fp32_form"] = r32
        forms["fp32_form"] = c32
    if args.precision == "bf16" and not args.no_fp32:
        s8, r8, c8 = measure(timer, w, trace, blob32, "fp8", args.steps, args.warmup, rec, off,
                             autotune=not args.no_autotune, persistent=not args.layerwise)
        s8.close()
        r8["note"] = "FP8 e4m3 tcgen05 path, same workload and timing"
        k8 = PATH_KERNEL.get(r8["kernel_mode"], r8["kernel_mode"])
        r8["roofline"] = whole_call_roofline(w, "fp8", N, r8["ms_per_step"], k8, traffic_of(args, w.name, "fp8", k8))
        out["fp8_form"] = r8
        forms["fp8_form"] = c8
    if train_info:
        out["trained_predictor"] = train_info
    del rec, off

    # the larger configurations, each in its own record (the main line stays the
    # c2 workload): c5 at BF16 and FP8, c4 (trained predictor) at FP8 and BF16
    extra = {}
    if args.workload == "c2" and not args.no_extra and not args.subtrace_len:
        extra = run_extra(args, timer)
        out.update({k: v["record"] for k, v in extra.items()})

    # CPU side last (nothing on the GPU is timed while the oracle runs)
    if not args.no_cpu_baseline:
        blob64 = blob32.astype(np.float64) if train_info else I.workload_weights(w)
        if args.workload == "c4":   # the configuration's own check: 64 sampled sub-traces
            ids = sorted(np.random.default_rng(w.seed).choice(trace.n_subtraces, 64, replace=False).tolist())
            threads = host_cores()
        else:
            ids, threads = cpu_sample_ids(w, trace, blob64)
        rate, n, dt, r = oracle_rate(w, trace, blob64, ids, threads=threads)
        rate1, n1, dt1, _ = oracle_rate(w, trace, blob64, ids[:1], threads=1)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"{len(ids)} whole sub-traces ({n} instructions) of the same "
                                         f"workload, {dt:.1f} s, FP64",
                               "value_1_thread": rate1,
                               "sample_1_thread": f"1 whole sub-trace ({n1} instructions), {dt1:.1f} s",
                               "cpu_model": cpu_model(), "nproc": os.cpu_count()}
        out["cpi_error_vs_oracle"] = {"sampled_subtraces": len(ids), "cpi_error": cpi_error(cycles, ids, r.cycles)}
        for k, c in forms.items():
            out[k]["cpi_error_vs_oracle"] = {"sampled_subtraces": len(ids), "cpi_error": cpi_error(c, ids, r.cycles)}
        runs = {}   # one oracle run per workload (the precisions share its sample and weights)
        for k, v in extra.items():
            ew, etrace, eblob, eids = v["check"]
            if ew.name not in runs:
                runs[ew.name] = oracle_rate(ew, etrace, eblob, eids, threads=host_cores())
            _, en, edt, er = runs[ew.name]
            out[k]["cpi_error_vs_oracle"] = {"sampled_subtraces": len(eids), "instructions": en,
                                             "oracle_s": edt, "cpi_error": cpi_error(v["cycles"], eids, er.cycles)}
    print(json.dumps(out), flush=True)


def executed_work(w, prec, n_inst, ms_per_call, blob, rec, off):
    """The grid-persistent kernel computes only the positions below the padding
    extent: one more call with the kernel's row counters on gives the GEMM rows
    each layer computed, hence the executed FLOPs (conv1 with its 64 padded
    feature channels, FC2 from the instruction count)."""
    from paper_2105_05821_b300.simnet import Simnet
    a = w.arch
    sim = Simnet.for_arch(a, precision=prec, retire_width=w.retire_width, kernel_events=True, cluster=False)
    sim.load_weights(blob.astype(np.float32))
    sim.simulate(rec, off, stats=True)
    d = sim.phase_detail(8).reshape(-1)   # 8 x 4 counters from the persistent block
    sim.close()
    rows = [int(x) for x in d[24:24 + a.n_conv + 1]]
    exe = 0.0
    for l in range(a.n_conv):
        k = 2 * 64 if l == 0 else 2 * a.channels
        exe += 2.0 * rows[l] * k * a.channels
    exe += 2.0 * rows[a.n_conv] * a.channels * a.hidden   # FC1: last-layer positions x slots
    exe += 2.0 * a.n_out * a.hidden * n_inst              # FC2
    _, _, bf16_sus, src = peaks()
    peak = bf16_sus * (2.0 if prec == "fp8" else 1.0)
    tf = exe / (ms_per_call / 1e3) / 1e12
    return {"executed_flop": exe, "executed_tflops": tf, "executed_frac": tf / peak,
            "executed_note": f"GEMM rows per layer {rows} (output positions x active slots over the call, "
                             f"FC1: last-layer positions x slots) from the kernel's counters; frac against "
                             f"the {src} sustained peak" + (" x2" if prec == "fp8" else "")}


def run_extra(args, timer):
    """c5 (65,536 sub-traces, 100M instructions, W=128, 5 x Conv256, FC1024) at
    BF16 and FP8, and c4 (4,096 log-normal sub-traces, about 40M instructions,
    the trained c2 architecture) at FP8 and BF16.  Each record: inst/s, ms per
    call, the roofline of the whole call, and (filled in later) the CPI error
    of the sampled sub-traces against the FP64 oracle."""
    import torch
    res = {}
    steps, warmup = max(2, args.extra_steps), 1
    w5 = I.WORKLOADS["c5"]
    t5 = I.make_trace(w5)
    b5 = I.workload_weights(w5)
    ids5 = sorted(np.random.default_rng(w5.seed).choice(t5.n_subtraces, args.c5_sample, replace=False).tolist())
    _, _, rec, off = device_trace(t5, timer.dev)
    for prec in ("bf16", "fp8"):
        sim, r, c = measure(timer, w5, t5, b5.astype(np.float32), prec, steps, warmup, rec, off)
        sim.close()
        r["workload"] = f"c5: {w5.description}; weights: {I.weight_recipe(w5)}"
        r["roofline"] = whole_call_roofline(w5, prec, t5.n_instructions, r["ms_per_step"],
                                            PATH_KERNEL.get(r["kernel_mode"], r["kernel_mode"]),
                                            traffic_of(args, "c5", prec, PATH_KERNEL.get(r["kernel_mode"])))
        if r["kernel_mode"] == "persistent":
            r["roofline"].update(executed_work(w5, prec, t5.n_instructions, r["ms_per_step"], b5, rec, off))
        res[f"c5_{prec}"] = {"record": r, "cycles": c, "check": (w5, t5, b5, ids5)}
    del rec, off
    torch.cuda.empty_cache()
    w4 = I.WORKLOADS["c4"]
    t4 = I.make_trace(w4)
    b4, info = train_predictor(w4, args.train_steps)
    ids4 = sorted(np.random.default_rng(w4.seed).choice(t4.n_subtraces, 64, replace=False).tolist())
    _, _, rec, off = device_trace(t4, timer.dev)
    for prec in ("fp8", "bf16"):
        sim, r, c = measure(timer, w4, t4, b4, prec, steps, warmup, rec, off, autotune=not args.no_autotune)
        sim.close()
        r["workload"] = f"c4: {w4.description}; {t4.n_instructions} instructions; trained predictor"
        r["trained_predictor"] = info
        r["roofline"] = whole_call_roofline(w4, prec, t4.n_instructions, r["ms_per_step"],
                                            PATH_KERNEL.get(r["kernel_mode"], r["kernel_mode"]))
        res[f"c4_{prec}"] = {"record": r, "cycles": c, "check": (w4, t4, b4.astype(np.float64), ids4)}
    del rec, off
    torch.cuda.empty_cache()
    return res


CLUSTER_PHASES = ["step start", "feature rows", "wait conv1", "epilogue conv1", "wait conv2", "epilogue conv2",
                  "wait conv3", "epilogue conv3", "wait FC1", "FC1 epilogue", "wait partials", "head", "extent"]


def cluster_phases(w, args, blob32, rec, off, sm_mhz):
    """CTA 0's time per phase of the cluster kernel (SM clock cycles of one
    extra timed call, converted at the sampled SM clock), in microseconds per
    lock-step."""
    import torch
    from paper_2105_05821_b300.simnet import Simnet
    cyc = torch.empty(off.numel() - 1, dtype=torch.int64, device=off.device)
    sim = Simnet.for_arch(w.arch, precision=args.precision, retire_width=w.retire_width, kernel_events=True)
    sim.load_weights(blob32)
    sim.simulate(rec, off, cycles_out=cyc, stats=True)
    d = sim.phase_detail(8).reshape(-1)
    sim.close()
    steps = max(int(d[14]), 1)
    names = [n for n in CLUSTER_PHASES]
    if w.arch.n_conv == 2:   # the third conv layer's slots stay empty
        names = names[:6] + ["-", "-"] + names[8:]
    out = {n: float(d[k]) / steps / sm_mhz for k, n in enumerate(names) if n != "-"}
    out["positions_per_step"] = float(d[15]) / steps
    # part of the last layer's wait: every CTA done reading the previous pass's exchanged rows
    out["wait exchange buffer free"] = float(d[13]) / steps / sm_mhz
    # the MMA warp's view of the same steps (counters 16-29 of the kernel; 30-31 are the
    # workers' FC1 epilogue)
    L = w.arch.n_conv
    detail = {"wait feature rows": 16, "wait extent": 17, "wait peer rows": 18, "FC1 issue": 19,
              "wait FC1 operand halves": 20, "FC1 epilogue arithmetic": 30, "partial sums sent": 31}
    for l in range(L):
        if l > 0:
            detail[f"wait conv{l + 1} operand halves"] = 20 + l
        detail[f"conv{l + 1} issue"] = 23 + l
        detail[f"conv{l + 1} weight waits"] = 26 + l
    detail["FC1 weight waits"] = 26 + L
    out["mma_warp"] = {n: float(d[k]) / steps / sm_mhz for n, k in detail.items()}
    return out


def roofline(w, args, blob32, rec, off, B, path):
    """Per-kernel CUDA-event times from one extra full step with an event pair
    around every launch; roofline of the kernel with the largest share."""
    import torch
    from paper_2105_05821_b300.simnet import Simnet
    cyc = torch.empty(B, dtype=torch.int64, device=off.device)
    hbm, bf16_burst, bf16_sus, src = peaks()
    # the per-layer or grid-persistent path the timed call finished on (a cluster
    # call that hands its long queues on is measured here as the path it moved to)
    sim = Simnet.for_arch(w.arch, precision=args.precision, retire_width=w.retire_width,
                          kernel_events=True, persistent=not args.layerwise and path != "layerwise",
                          cluster=False)
    sim.load_weights(blob32)
    if args.precision != "fp32" and not args.no_autotune:
        sim.autotune(B)
    sim.simulate(rec, off, cycles_out=cyc, stats=True)
    ms, n = sim.kernel_times()
    # the persistent kernel runs conv1 and conv2 of a 256-channel CNN as one phase,
    # timed under conv2's kind (conv1's kind then has no phases); CTA 0 sums that
    # phase's waits in conv1's row of the phase detail
    fused = n[1] == 0 and n[2] > 0
    waits = None
    if fused:
        d = sim.phase_detail(2)
        waits = {"mma_warp_free_accumulator": d[0][0] / 1e6, "mma_warp_operand_unit": d[0][1] / 1e6,
                 "mma_warp_a_operand_quarter": d[0][2] / 1e6, "epilogue_full_accumulator": d[0][3] / 1e6,
                 "phase_to_last_mma_commit": d[1][1] / 1e6, "phase_to_epilogue_done": d[1][2] / 1e6}
    sim.close()
    total = sum(ms)
    steps = max(n[10], 1)   # head/update: one launch (or phase) a step

    def units(k):
        amt, unit, bound = algorithmic_units(w, k, B, args.precision)
        if fused and k == 2:
            amt += algorithmic_units(w, 1, B, args.precision)[0]
        return amt, unit, bound

    def name(k):
        return "conv1_conv2_gemms_one_phase" if fused and k == 2 else kind_name(w, k)

    kernels = {}
    for k in range(len(ms)):
        if n[k] == 0:
            continue
        amt, unit, bound = units(k)
        kernels[name(k)] = {"launches": n[k], "ms_total": ms[k], "share": ms[k] / total,
                            "avg_us": 1e3 * ms[k] / n[k], "bound": bound}
        if fused and k == 2:   # CTA 0's summed milliseconds
            kernels[name(k)]["cta0_ms"] = waits
    dom = max(range(len(ms)), key=lambda k: ms[k])
    amt, unit, bound = units(dom)
    # per launch: the kind's per-step work over its launches (or phases) a step
    amt = amt * steps / n[dom]
    avg_s = ms[dom] / n[dom] / 1e3
    if unit == "flop":
        achieved = amt / avg_s / 1e12
        if bound == "alu":
            peak, punit, note = FP32_FMA_PEAK_TFLOPS, "TFLOP/s", "FP32 FMA peak at max SM clock"
        else:
            scale = 2.0 if args.precision == "fp8" else 1.0
            peak, punit, note = bf16_sus * scale, "TFLOP/s", f"{src} bf16 sustained" + (
                " x2 (fp8 nominal ratio)" if scale > 1 else "")
    else:
        achieved = amt / avg_s / 1e9
        peak, punit, note = hbm, "GB/s", f"{src} HBM copy"
    traffic = traffic_of(args, w.name, args.precision, name(dom))
    roof = {"kernel": name(dom), "bound": bound, "achieved": achieved, "peak": peak,
            "unit": punit, "frac": achieved / peak, "peak_source": note, "traffic": traffic,
            "avg_launch_us": avg_s * 1e6, "algorithmic_per_launch": amt, "algorithmic_unit": unit,
            "share_of_step": ms[dom] / total, "steps_timed": steps}
    return roof, kernels


def run_sweep(args):
    """Sub-trace length against simulation error, the trade-off behind splitting
    a trace for parallel simulation (Sec. 3.3): one synthetic trace of N
    instructions with the c2 workload's record mix and CNN, simulated by the
    FP64 oracle as one sub-trace (the reference: no split), and split into
    equal contiguous sub-traces, both by the oracle (the method's own error
    from splitting: every sub-trace starts from an empty queue and ends with
    its own drain) and on the GPU's default BF16 path (that error plus the
    precision's).  The GPU FP32 form of the unsplit trace is reported beside
    the oracle's.  Prints one JSON line."""
    import torch
    from paper_2105_05821_b300.simnet import Simnet
    import oracle
    w = I.WORKLOADS["c2"]
    N = args.sweep_n
    records = I.make_records(N, 7)
    blob64 = I.workload_weights(w)
    blob = blob64.astype(np.float32)
    cfg = oracle.Config.of(w.arch, retire_width=w.retire_width)
    rec = torch.from_numpy(records.view(np.int32).copy()).cuda()

    def gpu(sim, n_sub):
        off = torch.from_numpy(I.equal_offsets(N, n_sub)).cuda()
        sim.simulate(rec, off, stats=False)   # warm
        torch.cuda.synchronize()
        st = sim.simulate(rec, off)
        return st.total_cycles / N, st.ms_total, sim.kernel_path

    def orc(n_sub):
        t0 = time.perf_counter()
        r = oracle.simulate(cfg, records, I.equal_offsets(N, n_sub), blob64, n_threads=host_cores())
        return float(r.cycles.sum()) / N, time.perf_counter() - t0

    cpi_ref, s_ref = orc(1)
    ref32 = Simnet.for_arch(w.arch, precision="fp32", retire_width=w.retire_width)
    ref32.load_weights(blob)
    cpi32, ms32, _ = gpu(ref32, 1)
    sim = Simnet.for_arch(w.arch, precision="bf16", retire_width=w.retire_width)
    sim.load_weights(blob)
    rows = []
    length = N
    while length >= args.sweep_min:
        n_sub = N // length
        cpi, ms, path = gpu(sim, n_sub)
        cpi_o, s_o = (cpi_ref, s_ref) if n_sub == 1 else orc(n_sub)
        rows.append({"subtrace_len": length, "n_subtraces": n_sub, "cpi_gpu_bf16": cpi,
                     "cpi_oracle_split": cpi_o, "split_error_oracle": cpi_o / cpi_ref - 1.0,
                     "gpu_error_vs_oracle_unsplit": cpi / cpi_ref - 1.0,
                     "gpu_error_vs_oracle_split": cpi / cpi_o - 1.0, "oracle_s": s_o,
                     "ms": ms, "inst_per_s": N / (ms / 1e3), "kernel_mode": path})
        length //= 4
    print(json.dumps({"metric": "CPI error of split simulation vs sub-trace length", "unit": "relative",
                      "instructions": N, "data": "synthetic",
                      "reference": {"form": "FP64 oracle, one sub-trace", "cpi": cpi_ref, "oracle_s": s_ref},
                      "gpu_fp32_unsplit": {"cpi": cpi32, "error_vs_oracle": cpi32 / cpi_ref - 1.0, "ms": ms32},
                      "rows": rows}))


def run_training(args):
    """Training throughput on the training workload (windows/s of fused library
    steps: gather, forward, loss, hand-written backward, Adam; BF16 on the
    tensor cores, with the FP32 CUDA-core form beside it); a side measurement,
    not the simulation metric."""
    import torch
    from paper_2105_05821_b300.simnet import Simnet
    from paper_2105_05821_b300.train import Windows
    w = I.WORKLOADS["c3"]
    rec = I.make_records(w.n_instructions, w.seed)
    labels = I.toy_labels(rec)
    win = Windows.from_labels(rec, labels)
    blob = I.workload_weights(w)
    batch = 4096
    g = torch.Generator(device="cuda").manual_seed(0)
    idx = [torch.randint(0, len(win), (batch,), device="cuda", generator=g) for _ in range(args.warmup + args.steps)]

    def one(prec):
        sim = Simnet.for_arch(w.arch, precision=prec)
        sim.load_weights(blob.astype(np.float32))
        for i in range(args.warmup):
            sim.train_step(win, idx[i], 1e-3)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for i in range(args.steps - 1):
            sim.train_step(win, idx[args.warmup + i], 1e-3, loss=False)
        last = sim.train_step(win, idx[args.warmup + args.steps - 1], 1e-3)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        sim.close()
        return {"value": batch / (ms / 1e3), "unit": "windows/s", "ms_per_step": ms, "loss_last": last,
                "dtype": prec}

    main = one(args.precision if args.precision != "fp8" else "bf16")
    out = {"metric": "training windows/s (fused gather, forward, loss, backward, Adam)", **main, "batch": batch,
           "steps": args.steps, "warmup": args.warmup,
           "config": {"workload": f"c3: {w.description}; weights: {I.weight_recipe(w)}"}}
    if main["dtype"] != "fp32":
        out["fp32_form"] = one("fp32")
        flop = 2.0 * 3.0 * w.arch.macs_per_inference() * batch     # forward, input and weight gradients
        hbm, burst, sus, src = peaks()
        out["roofline"] = {"bound": "tensor", "achieved": flop / (main["ms_per_step"] / 1e3) / 1e12,
                           "peak": sus, "unit": "TFLOP/s", "peak_source": f"{src} bf16 sustained",
                           "note": "3 x forward MACs per window (forward, input and weight gradients)"}
        out["roofline"]["frac"] = out["roofline"]["achieved"] / sus
    if not args.no_cpu_baseline:
        import oracle
        cfg = oracle.Config.of(w.arch)
        ids = np.random.default_rng(3).integers(0, len(rec), 64)
        x = oracle.window_features(cfg, rec, labels.fetch, labels.E, labels.ctx_begin, ids)
        y = np.stack([labels.F[ids], labels.E[ids]], 1).astype(np.float64)
        t0 = time.perf_counter()
        oracle.loss_grad(cfg, blob, x, y)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(ids) / dt, "unit": "windows/s", "cores": 1, "kind": "oracle",
                               "sample": f"FP64 forward + backward of {len(ids)} windows, {dt:.2f} s"}
    print(json.dumps(out), flush=True)


def main():
    faulthandler.enable()
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "rb7"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cluster", action="store_true", help="BF16: the grid-wide persistent kernel")
    ap.add_argument("--fixed-path", action="store_true",
                    help="no timed persistent / per-layer choice and no cluster probe: the path the flags select")
    ap.add_argument("--layerwise", action="store_true",
                    help="BF16/FP8: one kernel per layer and step instead of the persistent kernel")
    ap.add_argument("--head", default="regression", choices=["regression", "hybrid"],
                    help="latency head: regression (2 FC2 outputs) or the hybrid classes + regression (22)")
    ap.add_argument("--store-queue", action="store_true",
                    help="store latency and memory write queue (three latencies per instruction)")
    ap.add_argument("--untrained", action="store_true", help="c4: keep the seeded weights")
    ap.add_argument("--train-steps", type=int, default=300, help="c4: training steps before simulating")
    ap.add_argument("--sweep", action="store_true",
                    help="CPI error against sub-trace length (one trace split into more and more parts)")
    ap.add_argument("--sweep-n", type=int, default=65536, help="--sweep: trace length")
    ap.add_argument("--sweep-min", type=int, default=64, help="--sweep: shortest sub-trace")
    ap.add_argument("--no-extra", action="store_true",
                    help="c2: skip the c5 / c4 records (profiling runs)")
    ap.add_argument("--extra-steps", type=int, default=2, help="timed calls of each c5 / c4 record")
    ap.add_argument("--c5-sample", type=int, default=8, help="c5 sub-traces re-simulated by the oracle")
    ap.add_argument("--subtrace-len", type=int, default=0,
                    help="keep only the first N instructions of every sub-trace (profiling runs)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "c3":
        run_training(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if world > 1:
        # The simulation is built and measured on one GPU (its kernels use
        # thread-block clusters within one device and no collective).  Rank 0
        # says so; every rank exits without GPU work.
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "n_gpus": world,
                              "unavailable": "one GPU only: the simulation path is built and measured "
                                             "on a single B300 (run without torchrun)"}), flush=True)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
