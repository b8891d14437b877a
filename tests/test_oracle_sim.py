"""Pins of the oracle's queue/clock state machine and feature rows (no GPU).

Each test checks the FP64 oracle against something other than itself:
values stepped by hand (tests/golden/hand_trace.json), closed-form totals of a
constant stub predictor, a prefix-maximum formula of Eq. 1 for unbounded
retire bandwidth, and invariants of the queue (Sec. 3.1-3.3).
"""
import json
import math
import os

import numpy as np
import pytest
from hypothesis import given, settings, strategies as st

import oracle
from paper_2105_05821_b300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _hand():
    with open(os.path.join(GOLD, "hand_trace.json")) as f:
        g = json.load(f)
    cols = np.array(g["insts"]).T
    recs = I.pack_records(*cols)
    offs = np.array([0, len(recs)], np.int64)
    return g, recs, offs


@pytest.mark.parametrize("rule", ["ge", "gt"])
def test_hand_stepped_trace(rule):
    """Sec. 3.2 rules stepped by hand: clock, budgeted in-order retire, eviction, drain."""
    g, recs, offs = _hand()
    cfg = oracle.Config(window=g["window"], n_conv=1, channels=2, hidden=2,
                        retire_width=g["retire_width"], retire_strict=(rule == "gt"))
    r = oracle.simulate(cfg, recs, offs, replay=np.array(g["replay"], np.uint8), logs=True)
    exp = g[rule]
    assert r.tick.tolist() == exp["tick"]
    assert r.qlen.tolist() == exp["len"]
    assert int(r.evictions[0]) == exp["evictions"]
    assert int(r.cycles[0]) == exp["cycles"]
    # Eq. 1: final curTick = sum of F + Delta with Delta >= 1
    assert int(r.cycles[0]) == sum(f for f, _ in g["replay"]) + (exp["cycles"] - exp["tick"][-1])


def test_hand_features():
    """Feature rows (current + newest-first context) at two steps of the hand trace."""
    g, recs, offs = _hand()
    cfg = oracle.Config(window=g["window"], n_conv=1, channels=2, hidden=2,
                        retire_width=g["retire_width"])
    r = oracle.simulate(cfg, recs, offs, replay=np.array(g["replay"], np.uint8), features=True)
    for step in ("step2", "step3"):
        X = r.feat[int(step[-1])]
        exp = np.zeros_like(X)
        for row, ch in g["features"][step].items():
            for c, v in ch.items():
                exp[int(row[3:]), int(c)] = v
        np.testing.assert_array_equal(X, exp)


@pytest.mark.parametrize("n,f,e,window,rw", [
    (50, 1, 0, 8, 2), (50, 1, 5, 8, 1), (37, 2, 9, 8, 8), (200, 3, 30, 16, 4),
    (5, 1, 7, 16, 8), (1, 4, 0, 4, 1), (64, 7, 7, 4, 3), (100, 1, 3, 32, 8)])
def test_closed_form_positive_fetch(n, f, e, window, rw):
    """Constant stub F = f >= 1, E = e, queue capacity >= ceil(e/f)+1:
    total = n*f + max(e, 1) and nothing is evicted."""
    cap = window - 1
    assert cap >= math.ceil(e / f) + 1
    recs = I.make_records(n, 7)
    cfg = oracle.Config(window=window, n_conv=1, channels=2, hidden=2, retire_width=rw)
    rep = np.tile(np.array([f, e], np.uint8), (n, 1))
    r = oracle.simulate(cfg, recs, np.array([0, n]), replay=rep)
    assert int(r.cycles[0]) == n * f + max(e, 1)
    assert int(r.evictions[0]) == 0


@pytest.mark.parametrize("n,e,window,rw", [
    (3, 0, 8, 2), (7, 4, 8, 2), (40, 0, 8, 3), (40, 9, 16, 4), (1, 0, 4, 1), (300, 2, 32, 8)])
def test_closed_form_zero_fetch(n, e, window, rw):
    """F = 0 everywhere: no retire during the steps (budget 0), the queue fills and
    evicts, then drains RW per cycle from max(e,1):
    total = max(e,1) + ceil(min(n,cap)/RW) - 1, evictions = max(0, n - cap)."""
    cap = window - 1
    recs = I.make_records(n, 9)
    cfg = oracle.Config(window=window, n_conv=1, channels=2, hidden=2, retire_width=rw)
    rep = np.tile(np.array([0, e], np.uint8), (n, 1))
    r = oracle.simulate(cfg, recs, np.array([0, n]), replay=rep)
    m = min(n, cap)
    assert int(r.cycles[0]) == max(e, 1) + -(-m // rw) - 1
    assert int(r.evictions[0]) == max(0, n - cap)


def test_empty_subtrace():
    cfg = oracle.Config(window=8, n_conv=1, channels=2, hidden=2)
    recs = I.make_records(10, 1)
    rep = np.ones((10, 2), np.uint8)
    r = oracle.simulate(cfg, recs, np.array([0, 0, 10, 10]), replay=rep)
    assert r.cycles.tolist() == [0, 10 + 1, 0]


lat = st.tuples(st.integers(0, 6), st.integers(0, 40))


@settings(max_examples=60, deadline=None)
@given(st.lists(lat, min_size=1, max_size=60))
def test_unbounded_retire_prefix_max(ls):
    """With retire bandwidth larger than any queue and no eviction, entry j leaves
    at the first step with F > 0 (or drain cycle) whose tick reaches
    max_{k<=j}(T_k + E_k); so the total is max(T_last + 1, max_j(T_j + E_j)) and
    the queue length after step i counts the entries not yet released."""
    n = len(ls)
    F = np.array([a for a, _ in ls], np.int64)
    E = np.array([b for _, b in ls], np.int64)
    T = np.cumsum(F)
    cfg = oracle.Config(window=128, n_conv=1, channels=2, hidden=2, retire_width=127)
    r = oracle.simulate(cfg, I.make_records(n, 3), np.array([0, n]),
                        replay=np.stack([F, E], 1).astype(np.uint8), logs=True)
    assert int(r.cycles[0]) == max(T[-1] + 1, int((T + E).max()))
    need = np.maximum.accumulate(T + E)             # tick at which entry j may leave
    for i in range(n):
        steps = [k for k in range(1, i + 1) if F[k] > 0]
        released = 0
        for j in range(i):
            if any(k > j and T[k] >= need[j] for k in steps):
                released += 1
        assert int(r.qlen[i]) == i + 1 - released
    assert (np.diff(r.tick) >= 0).all() and (r.tick == T).all()


@settings(max_examples=60, deadline=None)
@given(st.lists(lat, min_size=1, max_size=80), st.integers(2, 5), st.integers(1, 4),
       st.booleans())
def test_queue_invariants(ls, logw, rw, strict):
    """curTick is the running sum of F (clock rule), the queue never exceeds
    W-1 entries, evictions happen only at capacity, and the drain takes at least
    one and at most max(E) + ceil(cap/RW) cycles."""
    n = len(ls)
    window = 1 << logw
    cap = window - 1
    F = np.array([a for a, _ in ls], np.int64)
    E = np.array([b for _, b in ls], np.int64)
    cfg = oracle.Config(window=window, n_conv=1, channels=2, hidden=2, retire_width=rw,
                        retire_strict=strict)
    r = oracle.simulate(cfg, I.make_records(n, 5), np.array([0, n]),
                        replay=np.stack([F, E], 1).astype(np.uint8), logs=True)
    assert (r.tick == np.cumsum(F)).all()
    assert (r.qlen >= 1).all() and (r.qlen <= cap).all()
    delta = int(r.cycles[0]) - int(r.tick[-1])
    assert 1 <= delta <= int(E.max()) + int(strict) + -(-cap // rw)
    # an eviction is the only way the length fails to grow when nothing can retire (F = 0)
    ev = 0
    for i in range(1, n):
        if F[i] == 0:
            if r.qlen[i] == r.qlen[i - 1]:
                assert r.qlen[i - 1] == cap
                ev += 1
            else:
                assert r.qlen[i] == r.qlen[i - 1] + 1
    assert ev <= int(r.evictions[0])


def test_subtraces_independent_and_subset():
    """Sub-traces are simulated independently (Sec. 3.3): a subset run equals the
    same sub-traces of the full run, and permuting them changes nothing."""
    w = I.WORKLOADS["c1"]
    t = I.small_trace([40, 0, 17, 63, 25], seed=11)
    cfg = oracle.Config.of(w.arch)
    blob = I.workload_weights(w)
    full = oracle.simulate(cfg, t.records, t.offsets, blob, logs=True)
    sub = oracle.simulate(cfg, t.records, t.offsets, blob, subset=[3, 0], logs=True)
    assert sub.cycles.tolist() == [full.cycles[3], full.cycles[0]]
    a, b = t.offsets[3], t.offsets[4]
    np.testing.assert_array_equal(sub.lat[a:b], full.lat[a:b])
    # replaying the free-running latencies reproduces the run exactly
    rep = oracle.simulate(cfg, t.records, t.offsets, blob, replay=full.lat, logs=True)
    np.testing.assert_array_equal(rep.tick, full.tick)
    np.testing.assert_array_equal(rep.cycles, full.cycles)


def test_rounding_and_clamp():
    """Latency = softplus, clamped to [0, 255], rounded half to even; NaN -> 255.
    With all weights zero the output is softplus(FC2 bias); above 20 softplus is
    the identity, so the bias lands exactly on the rounding boundary."""
    arch = I.Arch(window=4, n_conv=1, channels=2, hidden=2)
    cfg = oracle.Config.of(arch, retire_width=1)
    n = oracle.blob_size(cfg)
    cases = [((22.5, 23.5), (22, 24)), ((300.0, -50.0), (255, 0)), ((0.0, 20.5), (1, 20)),
             ((float("nan"), 21.49999), (255, 21))]
    for (bf, be), (ef, ee) in cases:
        blob = np.zeros(n)
        blob[-2:] = (bf, be)
        r = oracle.simulate(cfg, I.make_records(3, 1), np.array([0, 3]), blob, logs=True)
        assert r.lat[:, 0].tolist() == [ef] * 3 and r.lat[:, 1].tolist() == [ee] * 3
