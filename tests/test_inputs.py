"""Host-side logic shared by the tests and the bench, checked without a GPU:
the packed instruction record (Sec. 2.2's per-instruction features in 26
bits), the workloads' sub-trace partitions, and the algorithmic FLOP count
per simulated instruction that every roofline figure divides by."""
import numpy as np
import pytest

import bench
from paper_2105_05821_b300 import inputs as I


FIELDS = [("opcode", 32), ("src0", 32), ("src1", 32), ("dst", 32), ("is_load", 2), ("is_store", 2),
          ("is_branch", 2), ("level", 3), ("mispredict", 2)]


def test_record_packing_round_trip_and_width():
    rng = np.random.default_rng(0)
    n = 4096
    cols = [rng.integers(0, hi, n) for _, hi in FIELDS]
    # every field also at its extremes, in one record each
    for j, (_, hi) in enumerate(FIELDS):
        cols[j][:2] = [0, hi - 1]
    r = I.pack_records(*cols)
    assert r.dtype == np.uint32
    assert int(r.max()) < (1 << 26)                 # 26 bits of record
    back = I.unpack_records(r)
    for (name, _), c in zip(FIELDS, cols):
        assert np.array_equal(back[name], c), name
    # each field alone with all of its bits set (widths 5, 5, 5, 5, 1, 1, 1, 2, 1) packs
    # to one contiguous run of bits, and the runs are disjoint and fill bits 0-25
    runs = 0
    for j, (name, width) in enumerate(zip([n for n, _ in FIELDS], [5, 5, 5, 5, 1, 1, 1, 2, 1])):
        one = [np.zeros(1, np.int64) for _ in FIELDS]
        one[j][0] = (1 << width) - 1
        v = int(I.pack_records(*one)[0])
        assert v != 0 and v & (v + (v & -v)) == 0, name      # contiguous
        assert runs & v == 0, name                            # disjoint
        runs |= v
    assert runs == (1 << 26) - 1


def test_equal_split_of_the_100m_trace():
    # 65,536 contiguous sub-traces of 100M instructions: 57,600 of 1,526 and 7,936 of 1,525
    off = I.equal_offsets(100_000_000, 65_536)
    lens = np.diff(off)
    assert off[0] == 0 and off[-1] == 100_000_000
    assert (lens[:57_600] == 1_526).all() and (lens[57_600:] == 1_525).all()


@pytest.mark.parametrize("b,n", [(1, 0), (3, 2), (8, 20_000), (1024, 1_024_000), (7, 100)])
def test_equal_offsets_cover_the_trace_contiguously(b, n):
    off = I.equal_offsets(n, b)
    lens = np.diff(off)
    assert len(off) == b + 1 and off[0] == 0 and off[-1] == n
    assert (lens >= 0).all() and lens.max() - lens.min() <= 1


def test_lognormal_lengths_stay_in_their_clip_and_are_seeded():
    w = I.WORKLOADS["c4"]
    a = I.lognormal_lengths(w.n_subtraces, w.seed, w.ln_median, w.ln_sigma, w.ln_clip)
    b = I.lognormal_lengths(w.n_subtraces, w.seed, w.ln_median, w.ln_sigma, w.ln_clip)
    assert np.array_equal(a, b)
    assert a.min() >= 1000 and a.max() <= 64000
    # median of a log-normal with median 8,000 (4,096 draws: within a few percent)
    assert abs(np.median(a) / 8000.0 - 1.0) < 0.05


def test_subset_keeps_each_subtrace_whole():
    t = I.small_trace([5, 0, 7, 3], seed=11)
    s = t.subset([2, 0, 1])
    assert list(s.lengths()) == [7, 5, 0]
    assert np.array_equal(s.records[:7], t.records[5:12])
    assert np.array_equal(s.records[7:12], t.records[0:5])


# Multiply-accumulates of one prediction, layer by layer, from the layer shapes
# (output positions x output channels x input channels x kernel 2 for a conv
# layer, inputs x outputs for a dense layer; the real 50 features, not the
# device padding to 64).
HAND_MACS = {
    "c1": [16 * 64 * 50 * 2, 8 * 64 * 64 * 2, 512 * 256, 256 * 2],
    "c2": [48 * 128 * 50 * 2, 24 * 128 * 128 * 2, 12 * 128 * 128 * 2, 1536 * 512, 512 * 2],
    "c5": [64 * 256 * 50 * 2, 32 * 256 * 256 * 2, 16 * 256 * 256 * 2, 8 * 256 * 256 * 2, 4 * 256 * 256 * 2,
           1024 * 1024, 1024 * 2],
}


@pytest.mark.parametrize("name,mflop", [("c1", 0.599), ("c2", 5.163), ("c5", 21.107)])
def test_flops_per_instruction(name, mflop):
    arch = I.WORKLOADS[name].arch
    macs = sum(HAND_MACS[name])
    assert arch.macs_per_inference() == macs
    assert round(2 * macs / 1e6, 3) == mflop


def test_whole_call_roofline_arithmetic():
    w = I.WORKLOADS["c2"]
    r = bench.whole_call_roofline(w, "bf16", 1_024_000, 10.0, "cluster_kernel", traffic=7.66e6)
    flops = 2 * sum(HAND_MACS["c2"]) * 1_024_000
    assert r["algorithmic_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / 0.010 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # a 10 ms call is held to the burst peak, FP8 to twice its BF16 figure
    _, burst, sustained, _ = bench.peaks()
    assert r["peak"] == pytest.approx(burst)
    r8 = bench.whole_call_roofline(w, "fp8", 1_024_000, 10.0, "cluster_kernel")
    assert r8["peak"] == pytest.approx(2 * burst)
    long = bench.whole_call_roofline(w, "bf16", 1_024_000, 1500.0, "persist_kernel")
    assert long["peak"] == pytest.approx(sustained)


def test_cpi_error_of_a_sample():
    gpu = np.array([100, 250, 75, 40])
    assert bench.cpi_error(gpu, [1, 3], np.array([250, 40])) == 0.0
    assert bench.cpi_error(gpu, [1, 3], np.array([290, 60])) == pytest.approx(abs(290 / 350 - 1.0))
