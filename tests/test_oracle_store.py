"""Pins of the oracle's memory write queue and store latency (Sec. 3.2), without
a GPU: hand-stepped traces (tests/golden/store_queue_trace.json), the
equivalences that must hold when no instruction is a store or every store's
latency is within its execution latency, the completion time of Eq. 1 when
retire bandwidth is unbounded, and the queue invariants."""
import json
import os

import numpy as np
import pytest
from hypothesis import given, settings, strategies as st

import oracle
from paper_2105_05821_b300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "store_queue_trace.json")))
STORE = 1 << 21


def cfg(window, rw=8, strict=False, store=True):
    return oracle.Config(window, 1, 8, 8, rw, strict, False, store)


def run(c, records, replay, features=False):
    rec = np.asarray(records, np.uint32)
    offs = np.array([0, len(rec)], np.int64)
    return oracle.simulate(c, rec, offs, replay=np.asarray(replay, np.uint8), logs=True, features=features)


@pytest.mark.parametrize("case", GOLD["cases"], ids=lambda k: k["name"])
def test_hand_stepped(case):
    c = cfg(case["window"], case["retire_width"], case["strict"])
    r = run(c, case["records"], case["replay"])
    assert r.cycles[0] == case["total"]
    assert r.evictions[0] == case["evictions"]
    np.testing.assert_array_equal(r.tick, case["tick"])
    np.testing.assert_array_equal(r.qlen, case["pq_len"])
    np.testing.assert_array_equal(r.mlen, case["wq_len"])
    np.testing.assert_array_equal(r.lat, case["replay"])


def test_hand_stepped_context_rows():
    case = GOLD["cases"][0]
    r = run(cfg(case["window"], case["retire_width"]), case["records"], case["replay"], features=True)
    for e in GOLD["features"]["rows"]:
        row = r.feat[e["step"], e["row"]]
        assert row[e["opcode"]] == 1.0 and row[:32].sum() == 1.0
        np.testing.assert_array_equal(row[42:45] * 64, e["ch42_43_44"])
    # rows past the context are zero; the current row has no latency features
    assert (r.feat[3, 3:] == 0).all() and (r.feat[:, 0, 42:50] == 0).all()


def random_case(rng, n, window, store_p):
    rec = I.make_records(n, int(rng.integers(1 << 30)))
    rec = (rec & ~np.uint32(STORE)) | np.where(rng.random(n) < store_p, STORE, 0).astype(np.uint32)
    lat = np.stack([rng.integers(0, 4, n), rng.integers(0, 12, n), rng.integers(0, 30, n)], 1)
    return rec, lat.astype(np.uint8)


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31), n=st.integers(1, 300), window=st.sampled_from([4, 8, 32]),
       rw=st.integers(1, 8), strict=st.booleans())
def test_without_stores_equals_the_processor_queue_alone(seed, n, window, rw, strict):
    rng = np.random.default_rng(seed)
    rec, lat = random_case(rng, n, window, 0.0)
    a = run(cfg(window, rw, strict, True), rec, lat)
    b = run(cfg(window, rw, strict, False), rec, lat[:, :2])
    np.testing.assert_array_equal(a.cycles, b.cycles)
    np.testing.assert_array_equal(a.evictions, b.evictions)
    np.testing.assert_array_equal(a.qlen, b.qlen)
    assert (a.mlen == 0).all()


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31), n=st.integers(1, 300), window=st.sampled_from([4, 8, 32]),
       rw=st.integers(1, 8), strict=st.booleans())
def test_stores_within_their_execution_latency_leave_at_once(seed, n, window, rw, strict):
    """S <= E: a store is already past its store latency when it retires from
    the processor queue, so the write queue is empty after every step and the
    timing equals the processor queue's alone."""
    rng = np.random.default_rng(seed)
    rec, lat = random_case(rng, n, window, 0.4)
    lat[:, 2] = np.minimum(lat[:, 2], lat[:, 1])
    a = run(cfg(window, rw, strict, True), rec, lat)
    b = run(cfg(window, rw, strict, False), rec, lat[:, :2])
    np.testing.assert_array_equal(a.cycles, b.cycles)
    np.testing.assert_array_equal(a.evictions, b.evictions)
    np.testing.assert_array_equal(a.qlen, b.qlen)
    assert (a.mlen == 0).all()


@settings(max_examples=60, deadline=None)
@given(seed=st.integers(0, 2**31), n=st.integers(1, 200), store_p=st.floats(0.0, 1.0))
def test_completion_time_with_unbounded_bandwidth(seed, n, store_p):
    """Eq. 1 with no retire limit and no eviction: the simulator empties at the
    first cycle after the last fetch by which every instruction is past its
    execution latency and every store past its store latency:
    total = max(T_n + 1, max_j T_j + E_j, max_{stores j} T_j + S_j)."""
    rng = np.random.default_rng(seed)
    rec, lat = random_case(rng, n, 256, store_p)
    lat[:, 0] = rng.integers(1, 4, n)            # F >= 1: every step has retire budget
    c = oracle.Config(256, 1, 8, 8, 255, False, False, True)
    r = run(c, rec, lat)
    T = np.cumsum(lat[:, 0].astype(np.int64))
    st_ = (rec & STORE) != 0
    expect = max(T[-1] + 1, int((T + lat[:, 1]).max()),
                 int((T + lat[:, 2])[st_].max()) if st_.any() else 0)
    assert r.cycles[0] == expect
    assert r.evictions[0] == 0


@settings(max_examples=30, deadline=None)
@given(seed=st.integers(0, 2**31), n=st.integers(1, 400), window=st.sampled_from([4, 8, 16]),
       rw=st.integers(1, 8))
def test_invariants(seed, n, window, rw):
    rng = np.random.default_rng(seed)
    rec, lat = random_case(rng, n, window, 0.5)
    r = run(cfg(window, rw), rec, lat)
    assert (r.qlen + r.mlen <= window - 1).all() and (r.qlen >= 1).all()
    stores_so_far = np.cumsum((rec & STORE) != 0)
    assert (r.mlen <= stores_so_far).all()                 # only stores enter the write queue
    assert (np.diff(r.tick) >= 0).all() and r.cycles[0] > r.tick[-1]
    # every instruction leaves: n = evicted + retired, and the drain is bounded
    assert r.cycles[0] - r.tick[-1] <= 255 + (window - 1) + 1 + 255


def test_cnn_store_output_drives_the_write_queue():
    """With the CNN, the third FC2 output is the store latency: FC2 reduced to
    its biases gives every instruction F = 1, E = 2, S = 7, which the stub path
    reproduces cycle for cycle."""
    arch = I.Arch(16, 2, 8, 12, store_queue=True)
    ws = I.he_weights(arch, 5)
    ws[-2] = ("fc2.weight", np.zeros((3, 12)))
    ws[-1] = ("fc2.bias", np.log(np.expm1(np.array([1.0, 2.0, 7.0]))))   # softplus^-1
    blob = I.flatten_weights(ws)
    c = oracle.Config.of(arch)
    assert c.store_queue and c.n_lat == 3 and c.n_out == 3 and oracle.blob_size(c) == arch.n_params()
    trace = I.small_trace([90, 33], seed=6)
    r = oracle.simulate(c, trace.records, trace.offsets, blob, logs=True)
    assert (r.lat == [1, 2, 7]).all()
    s = oracle.simulate(c, trace.records, trace.offsets, replay=r.lat, logs=True)
    np.testing.assert_array_equal(r.cycles, s.cycles)
    assert (r.mlen > 0).any()


@pytest.mark.parametrize("n,k", [(10, 6), (10, 20), (40, 3), (1, 1)])
def test_write_queue_has_no_retire_limit(n, k):
    """n stores fetched in one cycle (F = 1, then F = 0), E = 0, S = k, retire
    width 1: the drain moves one store a cycle into the write queue, and all
    stores past their store latency leave it together, so the simulator
    empties at 1 + max(k, n).  A write queue limited to one store a cycle
    would need 2k cycles for the first k."""
    rec = np.full(n, STORE, np.uint32) | np.arange(n, dtype=np.uint32) % 32
    lat = np.zeros((n, 3), np.uint8)
    lat[0, 0] = 1
    lat[:, 2] = k
    r = run(cfg(64, rw=1), rec, lat)
    assert r.cycles[0] == 1 + max(k, n)
