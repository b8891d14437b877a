"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and
the benchmark.

This module draws numbers and lays them out; it holds none of the simulation's
arithmetic.  Both the CUDA library and the FP64 oracle decode the 32-bit
instruction record below with code of their own.

Instruction record (one ``uint32`` per dynamic instruction)::

    bits  0-4   opcode class           (0..31)
    bits  5-9   source register 0      (0..31)
    bits 10-14  source register 1      (0..31)
    bits 15-19  destination register   (0..31)
    bit  20     is_load
    bit  21     is_store
    bit  22     is_branch
    bits 23-24  cache level            (0 = L1, 1 = L2, 2 = memory)
    bit  25     branch mispredict

The field distributions are the synthetic stand-ins for the gem5/SPEC traces
(Sec. 2.4, Table 1): opcode and registers uniform over 32, independent
Bernoulli flags (load 0.25, store 0.10, branch 0.15, mispredict 0.05) and a
cache level drawn for every instruction with p = (0.90, 0.08, 0.02).

Traces are split into contiguous sub-traces (Sec. 3.3): either equal sizes (the
first ``N mod B`` sub-traces take one more instruction) or log-normal lengths.
"""
from __future__ import annotations

import ctypes as _C
import os as _os
import subprocess as _sp
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np

N_FEATURES = 50          # features per instruction row (Sec. 2.2)
N_OPCODES = 32
N_REGS = 32
P_LOAD, P_STORE, P_BRANCH, P_MISPREDICT = 0.25, 0.10, 0.15, 0.05
P_LEVEL = (0.90, 0.08, 0.02)
CHUNK = 1 << 22          # instructions drawn per chunk; part of the stream's definition


# ----------------------------------------------------------------------------- workloads
@dataclass(frozen=True)
class Arch:
    """CNN shape: ``n_conv`` k=2/s=2 conv layers of ``channels`` outputs over
    ``window`` rows, then FC ``hidden`` and the output layer FC2 (Sec. 2.3).
    ``head`` = "regression": FC2 gives one value per latency (fetch,
    execution); "hybrid" (Sec. 2.3's hybrid scheme): per latency 10 class
    logits (0..8 cycles and "more than 8") and one regression value, in the
    order [fetch classes 0-9, fetch value, execution classes 0-9, execution
    value].  ``store_queue``: a third latency, the store latency (Sec. 2.2),
    after the other two, for the simulator's memory write queue (Sec. 3.2).
    ``block`` = "residual": the ``n_conv`` layers are residual blocks (the RB
    models of Sec. 2.3), each y = ReLU(pw(ReLU(conv(x))) + proj(x)) with conv
    and proj k=2 / stride-2 convolutions (proj without bias) and pw a
    pointwise (k=1) convolution."""
    window: int
    n_conv: int
    channels: int
    hidden: int
    head: str = "regression"
    store_queue: bool = False
    block: str = "conv"

    @property
    def n_lat(self) -> int:
        return 3 if self.store_queue else 2

    @property
    def n_out(self) -> int:
        return (11 if self.head == "hybrid" else 1) * self.n_lat

    @property
    def rows_out(self) -> int:
        return self.window >> self.n_conv

    @property
    def fc1_in(self) -> int:
        return self.channels * self.rows_out

    def shapes(self) -> List[Tuple[str, Tuple[int, ...]]]:
        """Parameter names and PyTorch shapes, in blob order."""
        out: List[Tuple[str, Tuple[int, ...]]] = []
        cin, C = N_FEATURES, self.channels
        for k in range(self.n_conv):
            if self.block == "residual":
                out.append((f"rb{k + 1}.conv.weight", (C, cin, 2)))
                out.append((f"rb{k + 1}.conv.bias", (C,)))
                out.append((f"rb{k + 1}.pw.weight", (C, C, 1)))
                out.append((f"rb{k + 1}.pw.bias", (C,)))
                out.append((f"rb{k + 1}.proj.weight", (C, cin, 2)))
            else:
                out.append((f"conv{k + 1}.weight", (C, cin, 2)))
                out.append((f"conv{k + 1}.bias", (C,)))
            cin = C
        out.append(("fc1.weight", (self.hidden, self.fc1_in)))
        out.append(("fc1.bias", (self.hidden,)))
        out.append(("fc2.weight", (self.n_out, self.hidden)))
        out.append(("fc2.bias", (self.n_out,)))
        return out

    def n_params(self) -> int:
        return int(sum(np.prod(s) for _, s in self.shapes()))

    def macs_per_inference(self) -> int:
        """Multiply-accumulates of one prediction on the real 50 features."""
        macs, cin, rows = 0, N_FEATURES, self.window
        for _ in range(self.n_conv):
            rows //= 2
            macs += rows * self.channels * cin * 2
            if self.block == "residual":      # projection shortcut and pointwise conv
                macs += rows * self.channels * cin * 2 + rows * self.channels * self.channels
            cin = self.channels
        macs += self.fc1_in * self.hidden + self.hidden * self.n_out
        return macs


@dataclass(frozen=True)
class Workload:
    name: str
    arch: Arch
    n_subtraces: int
    n_instructions: int            # total (equal split) or 0 for log-normal
    lengths: str = "equal"         # "equal" | "lognormal"
    seed: int = 0
    retire_width: int = 8          # O3CPU commit width (Table 2)
    ln_median: float = 8000.0
    ln_sigma: float = 0.63
    ln_clip: Tuple[int, int] = (1000, 64000)
    description: str = ""


ARCH_SMALL = lambda w: Arch(window=w, n_conv=2, channels=64, hidden=256)   # noqa: E731
ARCH_MID = Arch(window=96, n_conv=3, channels=128, hidden=512)
ARCH_WIDE = Arch(window=128, n_conv=5, channels=256, hidden=1024)
ARCH_RB7 = Arch(window=128, n_conv=7, channels=256, hidden=1024, head="hybrid", block="residual")

WORKLOADS: Dict[str, Workload] = {
    "c1": Workload("c1", ARCH_SMALL(32), 8, 20_000, seed=1,
                   description="8 sub-traces x 2,500 inst, W=32, 2xConv64, FC256"),
    "c2": Workload("c2", ARCH_MID, 1024, 1_024_000, seed=2,
                   description="1,024 sub-traces x 1,000 inst, W=96, 3xConv128, FC512"),
    "c3": Workload("c3", ARCH_SMALL(96), 1, 2_000_000, seed=3,
                   description="2M labelled windows, W=96, 2xConv64, FC256 (training)"),
    "c4": Workload("c4", ARCH_MID, 4096, 0, lengths="lognormal", seed=4,
                   description="4,096 sub-traces, log-normal lengths (median 8k, clip 1k-64k), W=96"),
    "c5": Workload("c5", ARCH_WIDE, 65_536, 100_000_000, seed=5,
                   description="65,536 sub-traces x ~1,526 inst (100M), W=128, 5xConv256, FC1024"),
    # the paper's most accurate model family: residual blocks with the hybrid head
    "rb7": Workload("rb7", ARCH_RB7, 1024, 1_024_000, seed=6,
                    description="1,024 sub-traces x 1,000 inst, W=128, 7 residual blocks of 256 channels, "
                                "FC1024, hybrid head"),
}


# ----------------------------------------------------------------------------- records
def pack_records(op, s0, s1, dst, ld, st, br, lvl, mp) -> np.ndarray:
    r = (op.astype(np.uint32)
         | (s0.astype(np.uint32) << 5)
         | (s1.astype(np.uint32) << 10)
         | (dst.astype(np.uint32) << 15)
         | (ld.astype(np.uint32) << 20)
         | (st.astype(np.uint32) << 21)
         | (br.astype(np.uint32) << 22)
         | (lvl.astype(np.uint32) << 23)
         | (mp.astype(np.uint32) << 25))
    return r.astype(np.uint32)


def unpack_records(r: np.ndarray) -> Dict[str, np.ndarray]:
    r = np.asarray(r, dtype=np.uint32)
    return {
        "opcode": (r & 31).astype(np.int64),
        "src0": ((r >> 5) & 31).astype(np.int64),
        "src1": ((r >> 10) & 31).astype(np.int64),
        "dst": ((r >> 15) & 31).astype(np.int64),
        "is_load": ((r >> 20) & 1).astype(np.int64),
        "is_store": ((r >> 21) & 1).astype(np.int64),
        "is_branch": ((r >> 22) & 1).astype(np.int64),
        "level": ((r >> 23) & 3).astype(np.int64),
        "mispredict": ((r >> 25) & 1).astype(np.int64),
    }


def make_records(n: int, seed: int) -> np.ndarray:
    """``n`` packed instruction records from numpy PCG64(seed), drawn in chunks of
    ``CHUNK`` instructions, fields in record order within each chunk."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty(n, dtype=np.uint32)
    for lo in range(0, n, CHUNK):
        m = min(CHUNK, n - lo)
        op = rng.integers(0, N_OPCODES, m, dtype=np.uint8)
        s0 = rng.integers(0, N_REGS, m, dtype=np.uint8)
        s1 = rng.integers(0, N_REGS, m, dtype=np.uint8)
        dst = rng.integers(0, N_REGS, m, dtype=np.uint8)
        ld = rng.random(m, dtype=np.float32) < P_LOAD
        st = rng.random(m, dtype=np.float32) < P_STORE
        br = rng.random(m, dtype=np.float32) < P_BRANCH
        u = rng.random(m, dtype=np.float32)
        lvl = (u >= P_LEVEL[0]).astype(np.uint8) + (u >= P_LEVEL[0] + P_LEVEL[1]).astype(np.uint8)
        mp = rng.random(m, dtype=np.float32) < P_MISPREDICT
        out[lo:lo + m] = pack_records(op, s0, s1, dst, ld, st, br, lvl, mp)
    return out


# ----------------------------------------------------------------------------- sub-traces
def equal_offsets(n: int, b: int) -> np.ndarray:
    """Offsets [b+1] of ``b`` contiguous sub-traces covering ``n`` instructions;
    the first ``n mod b`` take one instruction more."""
    base, extra = divmod(n, b)
    lens = np.full(b, base, dtype=np.int64)
    lens[:extra] += 1
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


def lognormal_lengths(b: int, seed: int, median: float, sigma: float,
                      clip: Tuple[int, int]) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 1_000_003))
    x = np.exp(rng.normal(np.log(median), sigma, b))
    return np.clip(np.rint(x), clip[0], clip[1]).astype(np.int64)


@dataclass
class Trace:
    records: np.ndarray            # uint32 [N]
    offsets: np.ndarray            # int64 [B+1]

    @property
    def n_subtraces(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_instructions(self) -> int:
        return int(self.offsets[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, ids) -> "Trace":
        """A trace holding only the listed sub-traces, in the given order."""
        ids = np.asarray(ids, dtype=np.int64)
        parts = [self.records[self.offsets[i]:self.offsets[i + 1]] for i in ids]
        lens = np.array([len(p) for p in parts], dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        recs = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
        return Trace(recs.astype(np.uint32), offs)


def make_trace(w: Workload, n_subtraces: int | None = None) -> Trace:
    """The workload's trace.  ``n_subtraces`` keeps only the first sub-traces
    (they are independent, so a prefix is a faithful sample)."""
    if w.lengths == "equal":
        offs = equal_offsets(w.n_instructions, w.n_subtraces)
    else:
        lens = lognormal_lengths(w.n_subtraces, w.seed, w.ln_median, w.ln_sigma, w.ln_clip)
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    if n_subtraces is not None:
        offs = offs[:n_subtraces + 1].copy()
    recs = make_records(int(offs[-1]), w.seed)
    return Trace(recs, offs)


def small_trace(lengths, seed: int) -> Trace:
    lens = np.asarray(lengths, dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return Trace(make_records(int(offs[-1]), seed), offs)


# ----------------------------------------------------------------------------- weights
def he_weights(arch: Arch, seed: int, bias_std: float = 0.0) -> List[Tuple[str, np.ndarray]]:
    """He-normal weights (std = sqrt(2 / fan_in), fan_in = C_in*2 for a conv,
    in_features for an FC) drawn from PCG64(seed) in blob order; biases are 0
    unless ``bias_std`` > 0, in which case they are drawn N(0, bias_std) after
    the weight they follow."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for name, shape in arch.shapes():
        if name.endswith("weight"):
            fan_in = shape[1] * (shape[2] if len(shape) == 3 else 1)
            out.append((name, rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)))
        else:
            b = rng.standard_normal(shape) * bias_std if bias_std > 0 else np.zeros(shape)
            out.append((name, b))
    return out


def flatten_weights(ws: List[Tuple[str, np.ndarray]], dtype=np.float64) -> np.ndarray:
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for _, a in ws]).astype(dtype)


def unflatten_weights(arch: Arch, blob: np.ndarray) -> List[Tuple[str, np.ndarray]]:
    out, k = [], 0
    for name, shape in arch.shapes():
        n = int(np.prod(shape))
        out.append((name, np.asarray(blob[k:k + n]).reshape(shape)))
        k += n
    assert k == len(blob), (k, len(blob))
    return out


FC2_GAIN = (8.0, 25.0, 25.0)    # scale of the fetch / execution / store rows of FC2
FC2_BIAS = (0.3, 12.0, 40.0)    # FC2 bias (fetch, execution, store)


# Hybrid head: class-logit rows are scaled by HYB_CLASS_GAIN and biased
# towards fetch latencies of 1-2 cycles and execution latencies of 3-8 cycles
# or "more than 8" (logit bias per class 0..9).  On the 1,024 x 1,000 workload
# the trajectory resembles the regression recipe's: CPI about 1.1-1.2 against
# 1.2, a queue about a tenth full, execution latencies split between the direct
# classes and the regression output (11-15 cycles).
HYB_CLASS_GAIN = 3.0
HYB_CLASS_BIAS = ((1.5, 3.5, 2.5, 1.0, -0.5, -1.0, -1.5, -2.0, -2.5, -3.0),
                  (-2.0, -0.5, 0.5, 1.0, 1.5, 1.5, 1.5, 1.5, 1.5, 2.5),
                  (-3.0, -2.0, -1.0, -0.5, 0.0, 0.0, 0.0, 0.5, 0.5, 3.0))   # store: mostly "more than 8"


def workload_weights(w: Workload) -> np.ndarray:
    """FP64 master blob for a workload: He-normal from PCG64(seed), zero
    biases, except that FC2's regression rows (fetch, execution, store) are scaled by
    ``FC2_GAIN`` and biased by ``FC2_BIAS``.  Plain He-init gives near-constant
    outputs (every F = 1, E = 0, a queue of length one); this recipe gives the
    mixed trajectory a trained predictor would (F mostly 0-1, E spread over
    1-20 cycles, the queue partly full, occasional evictions).  For a hybrid
    head the class-logit rows are scaled by ``HYB_CLASS_GAIN`` and biased by
    ``HYB_CLASS_BIAS`` (a mix of direct classes and the regression output)."""
    ws = he_weights(w.arch, w.seed)
    if w.arch.block == "residual":
        # the two branches of a block add: scale each by 1/sqrt(2) so that the
        # activations keep their size through the blocks
        ws = [(n, a / np.sqrt(2.0) if (n.endswith("pw.weight") or n.endswith("proj.weight")) else a)
              for n, a in ws]
    w2 = ws[-2][1].copy()
    b2 = np.zeros(w.arch.n_out)
    if w.arch.head == "hybrid":
        for t in range(w.arch.n_lat):
            w2[11 * t:11 * t + 10] *= HYB_CLASS_GAIN
            b2[11 * t:11 * t + 10] = HYB_CLASS_BIAS[t]
            w2[11 * t + 10] *= FC2_GAIN[t]
            b2[11 * t + 10] = FC2_BIAS[t]
    else:
        for t in range(w.arch.n_lat):
            w2[t] *= FC2_GAIN[t]
            b2[t] = FC2_BIAS[t]
    ws[-2] = ("fc2.weight", w2)
    ws[-1] = ("fc2.bias", b2)
    return flatten_weights(ws)


def weight_recipe(w: Workload) -> str:
    """One line naming the weight recipe of ``workload_weights``."""
    a = w.arch
    names = ("fetch", "execution", "store")[:a.n_lat]
    rows = ", ".join(f"{n} x{FC2_GAIN[t]:g} bias {FC2_BIAS[t]:g}" for t, n in enumerate(names))
    s = f"He-normal from PCG64(seed {w.seed}), zero biases; FC2 regression rows {rows}"
    if a.head == "hybrid":
        s += f"; class-logit rows x{HYB_CLASS_GAIN:g} with per-class biases"
    if a.block == "residual":
        s += "; residual branches scaled by 1/sqrt(2)"
    return s


# ----------------------------------------------------------------------------- random inputs
def random_windows(n: int, arch: Arch, seed: int) -> np.ndarray:
    """Feature matrices [n, W, 50] with the encoding's value set (one-hots,
    k/32 register ids, k/64 latencies), for CNN-only checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.zeros((n, arch.window, N_FEATURES))
    op = rng.integers(0, 32, (n, arch.window))
    np.put_along_axis(x[:, :, :32], op[..., None], 1.0, axis=2)
    x[:, :, 32:35] = rng.integers(0, 32, (n, arch.window, 3)) / 32.0
    x[:, :, 35:38] = rng.random((n, arch.window, 3)) < 0.2
    lvl = rng.integers(0, 3, (n, arch.window))
    np.put_along_axis(x[:, :, 38:41], lvl[..., None], 1.0, axis=2)
    x[:, :, 41] = rng.random((n, arch.window)) < 0.05
    x[:, :, 42] = rng.integers(0, 4096, (n, arch.window)) / 64.0
    x[:, :, 43] = rng.integers(0, 256, (n, arch.window)) / 64.0
    x[:, :, 45:49] = rng.random((n, arch.window, 4)) < 0.1
    x[:, 0, 42:] = 0.0
    return x


# ----------------------------------------------------------------------------- training labels
_TOY_SRC = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "toy_pipeline.c")
_TOY_LIB = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "libtoypipe.so")
_toy = None


def build_toy(force: bool = False) -> str:
    """Compile the toy pipeline timing model (gcc) next to its source."""
    if force or not _os.path.exists(_TOY_LIB) or _os.path.getmtime(_TOY_LIB) < _os.path.getmtime(_TOY_SRC):
        tmp = _TOY_LIB + f".tmp{_os.getpid()}"
        _sp.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _TOY_SRC])
        _os.replace(tmp, _TOY_LIB)
    return _TOY_LIB


@dataclass
class Labels:
    fetch: np.ndarray       # int64 [N] fetch cycle
    complete: np.ndarray    # int64 [N]
    commit: np.ndarray      # int64 [N]
    F: np.ndarray           # uint8 [N] fetch latency label
    E: np.ndarray           # uint8 [N] execution latency label
    ctx_begin: np.ndarray   # int64 [N] first context instruction of each window


def toy_labels(records: np.ndarray) -> Labels:
    """Run the toy 4-wide, 64-entry-ROB pipeline model over one trace."""
    global _toy
    if _toy is None:
        _toy = _C.CDLL(build_toy())
        _toy.toy_pipeline.restype = _C.c_int
        _toy.toy_pipeline.argtypes = [_C.c_void_p, _C.c_int64] + [_C.c_void_p] * 6
    rec = np.ascontiguousarray(records, dtype=np.uint32)
    n = len(rec)
    out = Labels(np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int64),
                 np.zeros(n, np.uint8), np.zeros(n, np.uint8), np.zeros(n, np.int64))
    p = lambda a: a.ctypes.data_as(_C.c_void_p)  # noqa: E731
    if _toy.toy_pipeline(p(rec), n, p(out.fetch), p(out.complete), p(out.commit), p(out.F), p(out.E),
                         p(out.ctx_begin)) != 0:
        raise MemoryError("toy_pipeline: allocation failed")
    return out
