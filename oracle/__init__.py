"""FP64 CPU oracle of SimNet's sub-trace simulation (ctypes binding of oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package and shares no code with it.

Functions follow SimNet (arXiv 2105.05821): features Sec. 2.2 / Table 1 (in a
synthetic encoding), CNN Sec. 2.3, queue and clock Sec. 3.2, Eq. 1 (Sec. 3.1),
independent sub-traces Sec. 3.3, squared-error training with Adam Sec. 2.4.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
NF = 50


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP) into liboracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("window", C.c_int32), ("n_conv", C.c_int32), ("channels", C.c_int32),
                ("hidden", C.c_int32), ("retire_width", C.c_int32), ("retire_strict", C.c_int32),
                ("hybrid", C.c_int32), ("store_queue", C.c_int32), ("residual", C.c_int32)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.oracle_blob_size.restype = C.c_int64
        _lib.oracle_blob_size.argtypes = [P]
        _lib.oracle_simulate.restype = C.c_int
        _lib.oracle_simulate.argtypes = [P, P, P, P, C.c_int32, P, C.c_int32, P, P, P,
                                         P, P, P, P, P, P, C.c_int32]
        _lib.oracle_cnn_forward.restype = C.c_int
        _lib.oracle_cnn_forward.argtypes = [P, P, P, C.c_int64, P, C.c_int32]
        _lib.oracle_head.restype = C.c_int
        _lib.oracle_head.argtypes = [P, P, C.c_int64, P, P]
        _lib.oracle_window_features.restype = C.c_int
        _lib.oracle_window_features.argtypes = [P, P, C.c_int64, P, P, P, P, C.c_int64, P]
        _lib.oracle_loss_grad.restype = C.c_int
        _lib.oracle_loss_grad.argtypes = [P, P, P, P, C.c_int64, P, P]
        _lib.oracle_adam.restype = None
        _lib.oracle_adam.argtypes = [P, P, P, P, C.c_int64, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_int64]
        _lib.oracle_num_threads.restype = C.c_int
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


@dataclass(frozen=True)
class Config:
    window: int
    n_conv: int
    channels: int
    hidden: int
    retire_width: int = 8
    retire_strict: bool = False
    hybrid: bool = False          # hybrid head (11 FC2 outputs per latency) instead of regression (1)
    store_queue: bool = False     # store latency + memory write queue (3 latencies instead of 2)
    residual: bool = False        # residual blocks (RB models) instead of plain conv layers

    @property
    def n_lat(self) -> int:
        return 3 if self.store_queue else 2

    @property
    def n_out(self) -> int:
        return (11 if self.hybrid else 1) * self.n_lat

    def c(self) -> _Cfg:
        return _Cfg(self.window, self.n_conv, self.channels, self.hidden, self.retire_width,
                    int(self.retire_strict), int(self.hybrid), int(self.store_queue), int(self.residual))

    @staticmethod
    def of(arch, retire_width: int = 8, retire_strict: bool = False) -> "Config":
        return Config(arch.window, arch.n_conv, arch.channels, arch.hidden, retire_width,
                      retire_strict, getattr(arch, "head", "regression") == "hybrid",
                      bool(getattr(arch, "store_queue", False)), getattr(arch, "block", "conv") == "residual")


def blob_size(cfg: Config) -> int:
    c = cfg.c()
    return int(_L().oracle_blob_size(C.byref(c)))


def num_threads() -> int:
    return int(_L().oracle_num_threads())


@dataclass
class SimResult:
    cycles: np.ndarray                 # int64 [n_subset]: final curTick of each sub-trace
    evictions: np.ndarray              # int64 [n_subset]
    lat: Optional[np.ndarray] = None   # uint8 [N, n_lat] F, E (, S) used (global positions)
    pre: Optional[np.ndarray] = None   # float64 [N, n_lat] softplus outputs before rounding
    tick: Optional[np.ndarray] = None  # int64 [N] curTick after each step
    qlen: Optional[np.ndarray] = None  # int32 [N] processor-queue length after each step
    feat: Optional[np.ndarray] = None  # float64 [N, W, 50]
    mlen: Optional[np.ndarray] = None  # int32 [N] memory-write-queue length after each step


def simulate(cfg: Config, records: np.ndarray, offsets: np.ndarray,
             weights: Optional[np.ndarray] = None, subset=None,
             replay: Optional[np.ndarray] = None, logs: bool = False,
             features: bool = False, n_threads: int = 0) -> SimResult:
    """Run the sequential simulator on each listed sub-trace independently."""
    records = np.ascontiguousarray(records, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n_sub = len(offsets) - 1
    N = int(offsets[-1])
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
    m = n_sub if sub is None else len(sub)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and len(w) != blob_size(cfg):
        raise ValueError(f"weight blob has {len(w)} values, config needs {blob_size(cfg)}")
    NL = cfg.n_lat
    rp = None if replay is None else np.ascontiguousarray(replay, dtype=np.uint8).reshape(N, NL)
    cyc = np.zeros(m, np.int64)
    ev = np.zeros(m, np.int64)
    lat = np.zeros((N, NL), np.uint8) if logs else None
    pre = np.full((N, NL), np.nan) if (logs and w is not None) else None
    tick = np.zeros(N, np.int64) if logs else None
    qlen = np.zeros(N, np.int32) if logs else None
    mlen = np.zeros(N, np.int32) if logs else None
    feat = np.zeros((N, cfg.window, NF)) if features else None
    c = cfg.c()
    rc = _L().oracle_simulate(C.byref(c), _p(w), _p(records), _p(offsets), n_sub, _p(sub), m,
                              _p(rp), _p(cyc), _p(ev), _p(lat), _p(pre), _p(tick), _p(qlen),
                              _p(mlen), _p(feat), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_simulate rejected its arguments")
    return SimResult(cyc, ev, lat, pre, tick, qlen, feat, mlen)


def cnn_forward(cfg: Config, weights: np.ndarray, x: np.ndarray, n_threads: int = 0) -> np.ndarray:
    """FC2 outputs z [n, n_out] (before softplus / the class decision) for
    feature matrices x [n, W, 50]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    assert x.shape[1:] == (cfg.window, NF)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    z = np.zeros((n, cfg.n_out))
    c = cfg.c()
    if _L().oracle_cnn_forward(C.byref(c), _p(w), _p(x), n, _p(z), int(n_threads)) != 0:
        raise ValueError("bad config")
    return z


def head(cfg: Config, z: np.ndarray):
    """The head's latency decision on FC2 outputs z [n, n_out]: (lat [n, n_lat]
    uint8, pre [n, n_lat] softplus of the regression output)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    n = z.shape[0]
    assert z.shape[1:] == (cfg.n_out,)
    lat = np.zeros((n, cfg.n_lat), np.uint8)
    pre = np.zeros((n, cfg.n_lat))
    c = cfg.c()
    if _L().oracle_head(C.byref(c), _p(z), n, _p(lat), _p(pre)) != 0:
        raise ValueError("bad config")
    return lat, pre


def softplus(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.float64)
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def window_features(cfg: Config, records, fetch, e_label, ctx_begin, idx) -> np.ndarray:
    records = np.ascontiguousarray(records, dtype=np.uint32)
    fetch = np.ascontiguousarray(fetch, dtype=np.int64)
    e_label = np.ascontiguousarray(e_label, dtype=np.uint8)
    ctx_begin = np.ascontiguousarray(ctx_begin, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    x = np.zeros((len(idx), cfg.window, NF))
    c = cfg.c()
    rc = _L().oracle_window_features(C.byref(c), _p(records), len(records), _p(fetch),
                                     _p(e_label), _p(ctx_begin), _p(idx), len(idx), _p(x))
    if rc != 0:
        raise ValueError("oracle_window_features rejected its arguments")
    return x


def loss_grad(cfg: Config, weights: np.ndarray, x: np.ndarray, y: np.ndarray):
    """(loss, grad) for labels y [n, n_lat]: mean squared error of softplus(z), plus the
    cross-entropy of the class logits for a hybrid head (oracle.c states the loss)."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, cfg.n_lat)
    g = np.zeros_like(w)
    loss = C.c_double(0.0)
    c = cfg.c()
    rc = _L().oracle_loss_grad(C.byref(c), _p(w), _p(x), _p(y), len(y), C.byref(loss), _p(g))
    if rc != 0:
        raise ValueError("oracle_loss_grad rejected its arguments")
    return float(loss.value), g


def adam(theta, m, v, g, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, t=1) -> None:
    """In-place Adam step on float64 arrays."""
    for a in (theta, m, v, g):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _L().oracle_adam(_p(theta), _p(m), _p(v), _p(g), len(theta), lr, beta1, beta2, eps, int(t))
