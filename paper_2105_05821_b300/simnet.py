"""Python binding of libsimnet's C ABI (include/simnet.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams; tensors are passed as raw pointers.  There
is no fallback: if libsimnet.so is missing or cannot load, importing the
binding's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimnet.so")

FP32, BF16, FP8 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8}
FLAG_RETIRE_STRICT = 0x1
FLAG_NO_GRAPH = 0x2
FLAG_KERNEL_EVENTS = 0x4
FLAG_NO_PDL = 0x8
FLAG_LAYERWISE = 0x10
FLAG_NO_CLUSTER = 0x20
FLAG_HYBRID_HEAD = 0x40
FLAG_STORE_QUEUE = 0x80
FLAG_RESIDUAL = 0x100
FLAG_FIXED_PATH = 0x200
FLAG_NO_FUSE = 0x400
MAX_GEMMS = 25          # GEMMs of the deepest CNN: 3 per residual block (up to 8) + FC1
PATHS = {0: "none", 1: "layerwise", 2: "persistent", 3: "cluster"}
KERNEL_KINDS = 12
KERNEL_GATHER, KERNEL_LAYER0, KERNEL_HEAD_UPDATE, KERNEL_COMPACT = 0, 1, 10, 11
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESTATE", 6: "EUNSUPPORTED"}

EXPORTS = ["simnet_abi_version", "simnet_init", "simnet_destroy", "simnet_last_error",
           "simnet_weight_count", "simnet_load_weights", "simnet_simulate", "simnet_cnn_forward",
           "simnet_kernel_times", "simnet_cnn_forward_noalloc", "simnet_noalloc_scratch_bytes",
           "simnet_gather_windows", "simnet_train_forward", "simnet_train_backward", "simnet_train_step",
           "simnet_set_weights_device", "simnet_get_weights", "simnet_phase_detail", "simnet_autotune",
           "simnet_simulate_steps", "simnet_state_save", "simnet_state_load", "simnet_kernel_path",
           "simnet_path_choice", "simnet_train_loss", "simnet_autotune_plan"]
STATE_KINDS = {"sim": 0, "train": 1}


class SimnetError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("window", C.c_int32), ("n_conv", C.c_int32), ("conv_channels", C.c_int32),
                ("fc_hidden", C.c_int32), ("retire_width", C.c_int32), ("precision", C.c_int32),
                ("flags", C.c_uint32), ("barrier_limit_us", C.c_int32), ("spin_limit_ns", C.c_int64)]


class _Trace(C.Structure):
    _fields_ = [("records", C.c_void_p), ("offsets", C.c_void_p), ("n_subtraces", C.c_int32),
                ("reserved", C.c_int32), ("n_instructions", C.c_int64)]


class _Stats(C.Structure):
    _fields_ = [("total_cycles", C.c_int64), ("instructions", C.c_int64), ("steps", C.c_int64),
                ("evictions", C.c_int64), ("kernel_launches", C.c_int64), ("ms_total", C.c_float),
                ("pending", C.c_int32), ("steps_done", C.c_int64)]


class _Windows(C.Structure):
    _fields_ = [("records", C.c_void_p), ("fetch", C.c_void_p), ("e_label", C.c_void_p),
                ("ctx_begin", C.c_void_p), ("labels", C.c_void_p), ("n_records", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load libsimnet.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_2105_05821_b300.build`")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.simnet_abi_version.restype = C.c_int32
        L.simnet_init.restype = C.c_int
        L.simnet_init.argtypes = [C.POINTER(_Config), C.POINTER(P)]
        L.simnet_destroy.restype = None
        L.simnet_destroy.argtypes = [P]
        L.simnet_last_error.restype = C.c_char_p
        L.simnet_last_error.argtypes = [P]
        L.simnet_weight_count.restype = C.c_int64
        L.simnet_weight_count.argtypes = [P]
        L.simnet_load_weights.restype = C.c_int
        L.simnet_load_weights.argtypes = [P, P, C.c_int64]
        L.simnet_simulate.restype = C.c_int
        L.simnet_simulate.argtypes = [P, C.POINTER(_Trace), P, P, P, P, C.POINTER(_Stats), P]
        L.simnet_cnn_forward.restype = C.c_int
        L.simnet_cnn_forward.argtypes = [P, P, P, C.c_int32, P]
        L.simnet_kernel_times.restype = C.c_int
        L.simnet_kernel_times.argtypes = [P, P, P, C.c_int32]
        L.simnet_cnn_forward_noalloc.restype = C.c_int
        L.simnet_cnn_forward_noalloc.argtypes = [P, P, P, C.c_int32, P]
        L.simnet_noalloc_scratch_bytes.restype = C.c_size_t
        L.simnet_noalloc_scratch_bytes.argtypes = []
        L.simnet_gather_windows.restype = C.c_int
        L.simnet_gather_windows.argtypes = [P, C.POINTER(_Windows), P, C.c_int32, P, P]
        L.simnet_train_forward.restype = C.c_int
        L.simnet_train_forward.argtypes = [P, P, P, C.c_int32, P]
        L.simnet_train_backward.restype = C.c_int
        L.simnet_train_backward.argtypes = [P, P, P, P]
        L.simnet_train_loss.restype = C.c_int
        L.simnet_train_loss.argtypes = [P, P, P, C.c_int32, P, P, P, P]
        L.simnet_train_step.restype = C.c_int
        L.simnet_train_step.argtypes = [P, C.POINTER(_Windows), P, C.c_int32, C.c_float, P, P]
        L.simnet_set_weights_device.restype = C.c_int
        L.simnet_set_weights_device.argtypes = [P, P, P]
        L.simnet_get_weights.restype = C.c_int
        L.simnet_get_weights.argtypes = [P, P]
        L.simnet_autotune_plan.restype = C.c_int
        L.simnet_autotune_plan.argtypes = [P, P, C.c_int32]
        L.simnet_autotune.restype = C.c_int
        L.simnet_autotune.argtypes = [P, C.c_int32, C.c_int32, P, P]
        L.simnet_phase_detail.restype = C.c_int
        L.simnet_phase_detail.argtypes = [P, P, C.c_int32]
        L.simnet_simulate_steps.restype = C.c_int
        L.simnet_simulate_steps.argtypes = [P, C.POINTER(_Trace), P, P, P, P, C.c_int64, C.c_int32,
                                            C.POINTER(_Stats), P]
        L.simnet_state_save.restype = C.c_int
        L.simnet_state_save.argtypes = [P, C.c_int32, P, C.POINTER(C.c_size_t), P]
        L.simnet_state_load.restype = C.c_int
        L.simnet_state_load.argtypes = [P, C.c_int32, P, C.c_size_t, P]
        L.simnet_kernel_path.restype = C.c_int32
        L.simnet_kernel_path.argtypes = [P]
        L.simnet_path_choice.restype = C.c_int
        L.simnet_path_choice.argtypes = [P, C.POINTER(C.c_float), C.POINTER(C.c_int32)]
        _lib = L
    return _lib


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class Stats:
    total_cycles: int
    instructions: int
    steps: int
    evictions: int
    kernel_launches: int
    ms_total: float
    pending: int = 0
    steps_done: int = 0


class Simnet:
    """One libsimnet context: a CNN shape, a precision and its loaded weights."""

    def __init__(self, window: int, n_conv: int, channels: int, hidden: int,
                 precision: str | int = "fp32", retire_width: int = 8, strict: bool = False,
                 graph: bool = True, spin_limit_ns: int = 0, kernel_events: bool = False,
                 pdl: bool = True, persistent: bool = True, barrier_limit_us: int = 0,
                 cluster: bool = True, hybrid: bool = False, store_queue: bool = False,
                 residual: bool = False, auto_path: bool = True, fuse: bool = True):
        L = lib()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        flags = ((FLAG_RETIRE_STRICT if strict else 0) | (0 if graph else FLAG_NO_GRAPH)
                 | (FLAG_KERNEL_EVENTS if kernel_events else 0) | (0 if pdl else FLAG_NO_PDL)
                 | (0 if persistent else FLAG_LAYERWISE) | (0 if cluster else FLAG_NO_CLUSTER)
                 | (FLAG_HYBRID_HEAD if hybrid else 0) | (FLAG_STORE_QUEUE if store_queue else 0)
                 | (FLAG_RESIDUAL if residual else 0) | (0 if auto_path else FLAG_FIXED_PATH)
                 | (0 if fuse else FLAG_NO_FUSE))
        self._cfg = _Config(window, n_conv, channels, hidden, retire_width, prec, flags, barrier_limit_us,
                            spin_limit_ns)
        self.window = window
        self.precision = prec
        self.hybrid = bool(hybrid)
        self.store_queue = bool(store_queue)
        self.n_lat = 3 if store_queue else 2                      # latencies per instruction
        self.n_out = (11 if hybrid else 1) * self.n_lat          # FC2 outputs per window
        h = C.c_void_p()
        st = L.simnet_init(C.byref(self._cfg), C.byref(h))
        if st != 0:
            raise SimnetError(st, "simnet_init rejected the config")
        self._h = h

    @classmethod
    def for_arch(cls, arch, **kw) -> "Simnet":
        kw.setdefault("hybrid", getattr(arch, "head", "regression") == "hybrid")
        kw.setdefault("store_queue", bool(getattr(arch, "store_queue", False)))
        kw.setdefault("residual", getattr(arch, "block", "conv") == "residual")
        return cls(arch.window, arch.n_conv, arch.channels, arch.hidden, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib().simnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise SimnetError(st, lib().simnet_last_error(self._h).decode())

    @property
    def weight_count(self) -> int:
        return int(lib().simnet_weight_count(self._h))

    def load_weights(self, blob: np.ndarray) -> None:
        """Canonical FP32 blob (host), PyTorch shapes in layer order."""
        w = np.ascontiguousarray(blob, dtype=np.float32)
        self._check(lib().simnet_load_weights(self._h, w.ctypes.data_as(C.c_void_p), len(w)))

    def simulate(self, records, offsets, cycles_out=None, lat_log=None, pre_log=None, replay=None,
                 stats: bool = True, stream=None, max_steps: Optional[int] = None,
                 resume: bool = False) -> Optional[Stats]:
        """Simulate the sub-traces.  records: cuda int32/uint32 [N]; offsets: cuda int64 [B+1];
        cycles_out: cuda int64 [B] (allocated if None and returned in .cycles).  With
        max_steps, run at most that many lock-steps; resume=True continues the held state."""
        import torch
        B = offsets.numel() - 1
        if cycles_out is None:
            cycles_out = torch.empty(B, dtype=torch.int64, device=offsets.device)
        self.cycles = cycles_out
        tr = _Trace(_ptr(records), _ptr(offsets), B, 0, records.numel())
        st = _Stats()
        self._check(lib().simnet_simulate_steps(self._h, C.byref(tr), _ptr(cycles_out), _ptr(lat_log),
                                                _ptr(pre_log), _ptr(replay),
                                                -1 if max_steps is None else int(max_steps), int(resume),
                                                C.byref(st) if stats else None, _stream(stream)))
        if not stats:
            return None
        return Stats(st.total_cycles, st.instructions, st.steps, st.evictions, st.kernel_launches,
                     st.ms_total, st.pending, st.steps_done)

    def state_save(self, kind: str = "sim", stream=None) -> bytes:
        """The context's simulation ("sim") or training ("train") state as bytes."""
        n = C.c_size_t(0)
        k = STATE_KINDS[kind]
        self._check(lib().simnet_state_save(self._h, k, None, C.byref(n), _stream(stream)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().simnet_state_save(self._h, k, buf, C.byref(n), _stream(stream)))
        return buf.raw[:n.value]

    def state_load(self, data: bytes, kind: str = "sim", stream=None) -> None:
        """Import a state written by state_save (resume with simulate(..., resume=True))."""
        buf = C.create_string_buffer(bytes(data), len(data))
        self._check(lib().simnet_state_load(self._h, STATE_KINDS[kind], buf, len(data), _stream(stream)))

    @property
    def kernel_path(self) -> str:
        """Kernel path of the last simulate call: layerwise, persistent or cluster."""
        return PATHS.get(int(lib().simnet_kernel_path(self._h)), "none")

    @property
    def path_choice(self) -> dict:
        """The last timed persistent / per-layer comparison: device ms of each over the
        same number of steps from the same state (zeros if none ran)."""
        ms = (C.c_float * 2)()
        n = C.c_int32()
        self._check(lib().simnet_path_choice(self._h, ms, C.byref(n)))
        return {"persistent_ms": float(ms[0]), "layerwise_ms": float(ms[1]), "steps": int(n.value)}

    def phase_detail(self, n_layers):
        """Per GEMM layer: summed ns to first data, last MMA, epilogue done, barrier passed (CTA 0)."""
        out = np.zeros(4 * n_layers, dtype=np.uint64)
        self._check(lib().simnet_phase_detail(self._h, out.ctypes.data_as(C.c_void_p), 4 * n_layers))
        return out.reshape(n_layers, 4)

    def autotune(self, n_subtraces: int, steps: int = 24, stream=None):
        """Pick per-layer tile widths for this batch size by timing; returns them."""
        out = (C.c_int32 * MAX_GEMMS)()    # one tile width per GEMM of the CNN
        self._check(lib().simnet_autotune(self._h, n_subtraces, steps, out, _stream(stream)))
        return list(out)

    def autotune_plan(self) -> dict:
        """The autotuner's last choice: batch size, path and launch shapes."""
        out = (C.c_int32 * (6 + MAX_GEMMS))()
        self._check(lib().simnet_autotune_plan(self._h, out, 6 + MAX_GEMMS))
        v = list(out)
        return {"batch": v[0], "path": PATHS.get(v[1], "none"), "cluster_size": v[2], "cluster_stage_bytes": v[3],
                "cluster_stages": v[4], "persist_stages": v[5], "tile_widths": [x for x in v[6:] if x]}

    def kernel_times(self):
        """(ms, launches) per kernel kind of the last simulate with kernel_events=True."""
        ms = (C.c_float * KERNEL_KINDS)()
        n = (C.c_int64 * KERNEL_KINDS)()
        self._check(lib().simnet_kernel_times(self._h, ms, n, KERNEL_KINDS))
        return list(ms), list(n)

    def cnn_forward_noalloc(self, x, z, stream=None):
        """cnn_forward using the library's fixed scratch array instead of allocated
        workspace (FP32 contexts; the caller provides z)."""
        self._check(lib().simnet_cnn_forward_noalloc(self._h, _ptr(x), _ptr(z), x.shape[0],
                                                     _stream(stream)))
        return z

    def cnn_forward(self, x, z=None, stream=None):
        """FC2 outputs [n, n_out] (before softplus and the hybrid class decision)
        for cuda float32 features [n, W, 50]."""
        import torch
        n = x.shape[0]
        assert x.is_contiguous() and x.dtype == torch.float32 and tuple(x.shape[1:]) == (self.window, 50)
        if z is None:
            z = torch.empty((n, self.n_out), dtype=torch.float32, device=x.device)
        self._check(lib().simnet_cnn_forward(self._h, _ptr(x), _ptr(z), n, _stream(stream)))
        return z

    # ------------------------------------------------------------------ training
    def _win(self, w) -> "_Windows":
        return _Windows(_ptr(w.records), _ptr(w.fetch), _ptr(w.e_label), _ptr(w.ctx_begin),
                        _ptr(w.labels), w.records.numel())

    def gather_windows(self, w, idx, stream=None):
        """Feature matrices [n, W, 50] of the windows idx (cuda int64) of a labelled trace."""
        import torch
        x = torch.empty((idx.numel(), self.window, 50), dtype=torch.float32, device=idx.device)
        win = self._win(w)
        self._check(lib().simnet_gather_windows(self._h, C.byref(win), _ptr(idx), idx.numel(), _ptr(x),
                                                _stream(stream)))
        return x

    def train_forward(self, x, stream=None):
        import torch
        z = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        self._check(lib().simnet_train_forward(self._h, _ptr(x), _ptr(z), x.shape[0], _stream(stream)))
        return z

    def train_backward(self, dz, grad=None, stream=None):
        import torch
        if grad is None:
            grad = torch.empty(self.weight_count, dtype=torch.float32, device=dz.device)
        self._check(lib().simnet_train_backward(self._h, _ptr(dz), _ptr(grad), _stream(stream)))
        return grad

    def train_loss(self, z, labels, grad_scale=None, loss=None, dz=None, stream=None):
        """The training loss on FC2 outputs z [n, n_out] against uint8 labels [n, 2]
        (device): fills `loss` (float [1]) and/or `dz` (float [n, n_out]),
        dz scaled by the device scalar `grad_scale` when given."""
        self._check(lib().simnet_train_loss(self._h, _ptr(z), _ptr(labels), z.shape[0], _ptr(grad_scale),
                                            _ptr(loss), _ptr(dz), _stream(stream)))
        return loss, dz

    def train_step(self, w, idx, lr=1e-3, stream=None, loss: bool = True) -> Optional[float]:
        """One fused step; returns the loss (the call then synchronises), or
        None with loss=False (asynchronous)."""
        win = self._win(w)
        out = C.c_float(0.0)
        self._check(lib().simnet_train_step(self._h, C.byref(win), _ptr(idx), idx.numel(), float(lr),
                                            C.byref(out) if loss else None, _stream(stream)))
        return float(out.value) if loss else None

    def set_weights_device(self, blob, stream=None):
        self._check(lib().simnet_set_weights_device(self._h, _ptr(blob), _stream(stream)))

    def get_weights(self) -> np.ndarray:
        out = np.zeros(self.weight_count, dtype=np.float32)
        self._check(lib().simnet_get_weights(self._h, out.ctypes.data_as(C.c_void_p)))
        return out
