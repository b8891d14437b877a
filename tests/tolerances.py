"""The parity bounds of the CUDA path against the FP64 oracle: one row per
precision, asserted by every GPU test and by `smoke()`.

Latency error is the paper's prediction-error form |f - y| / (y + 1)
(Sec. 2.5), taken on the softplus outputs before clamping and rounding, GPU
against oracle on the same integer state (teacher forcing).  `LAT_MAX` bounds
every predicted latency of a test, `LAT_P99` the 99th percentile of them.
CNN outputs (FC2, before softplus) are held to the same bounds, element by
element, in the same form.  `CPI` bounds |CPI_gpu / CPI_oracle - 1| of a
free-running simulation (each side on its own trajectory).

FP32 is held to 1e-3.  BF16 and FP8 bound what their rounding gives on the
workloads' weights: the FC2 rows of the execution and store latencies carry
gains of 25 (the synthetic weight recipe; a trained predictor's FC2 rows are
larger still, its labels reaching 200+ cycles), so a rounding error of a few
hundredths of a unit in FC1's output moves those logits by one or more;
softplus is 1-Lipschitz, so a latency moves by at most as much, which is a
large relative error where the latency itself is near zero.  The largest
errors seen over all workloads, heads and kernel paths of the tests are inside
these rows: BF16 0.094-0.13 with a 99th percentile of 0.017-0.020 (c4,
trained predictor), 0.063 (store-queue workload), 0.010 (c5), 0.005 (c2);
FP8 1.6-3.4 with a 99th percentile of 0.26-0.29 (c4, trained predictor: the
training's float atomics make its weights, and these figures, differ from
run to run), 0.98 (store-queue workload), 0.14 (c5), 0.09 (c2).  The CPI row
holds for all of them (largest seen: BF16 0.007 on c5, FP8 0.017 on c4).
"""
import numpy as np

LAT_MAX = {"fp32": 1e-3, "bf16": 0.2, "fp8": 5.0}
LAT_P99 = {"fp32": 1e-3, "bf16": 0.03, "fp8": 0.5}
CPI = {"fp32": 1e-3, "bf16": 0.02, "fp8": 0.05}


def rel_error(gpu, ref):
    """|f - y| / (|y| + 1), element by element."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(gpu - ref) / (np.abs(ref) + 1.0)


def check(err, precision, what=""):
    """Assert the precision's row on a set of errors; returns (p50, p99, max)."""
    err = np.asarray(err, dtype=np.float64).reshape(-1)
    assert np.isfinite(err).all(), what
    if err.size == 0:
        return 0.0, 0.0, 0.0
    p50, p99, mx = float(np.median(err)), float(np.percentile(err, 99)), float(err.max())
    print(f"\n{what} {precision}: p50 {p50:.2e} p99 {p99:.2e} max {mx:.2e}")
    assert mx <= LAT_MAX[precision], (what, precision, "max", mx)
    assert p99 <= LAT_P99[precision], (what, precision, "p99", p99)
    return p50, p99, mx


def check_cpi(cpi_err, precision, what=""):
    print(f"\n{what} {precision}: CPI error {cpi_err:.2e}")
    assert cpi_err <= CPI[precision], (what, precision, cpi_err)
