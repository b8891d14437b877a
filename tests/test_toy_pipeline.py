"""The toy pipeline timing model that labels training windows, checked on
small traces worked by hand (4-wide fetch/issue/commit, 64-entry ROB, cache
latencies 4/14/200, 15-cycle mispredict penalty)."""
import numpy as np

from paper_2105_05821_b300 import inputs as I


def rec(op=0, s0=0, s1=0, dst=0, ld=0, st=0, br=0, lvl=0, mp=0):
    return int(I.pack_records(*[np.array([v]) for v in (op, s0, s1, dst, ld, st, br, lvl, mp)])[0])


def test_independent_alu_ops_fill_fetch_and_issue_width():
    # five 1-cycle ops on disjoint registers: 4 fetched in cycle 0, the fifth in cycle 1
    r = np.array([rec(0, 10 + i, 20 + i, i + 1) for i in range(5)], np.uint32)
    L = I.toy_labels(r)
    assert L.fetch.tolist() == [0, 0, 0, 0, 1]
    assert L.complete.tolist() == [2, 2, 2, 2, 3]     # issue at fetch + 1, latency 1
    assert L.commit.tolist() == [2, 2, 2, 2, 3]
    assert L.F.tolist() == [0, 0, 0, 0, 1] and L.E.tolist() == [2] * 5
    assert L.ctx_begin.tolist() == [0, 0, 0, 0, 0]


def test_load_dependency_chain():
    # i0: L2 load (op 1) -> r1: 1 + 1 + 14 = 16 cycles, issue at 1, done 17
    # i1: op 2 reads r1 -> waits for 17, latency 3, done 20
    # i2: independent op 0 (1 cycle), done 2, but commits in order after i1 at 20
    r = np.array([rec(1, 5, 6, 1, ld=1, lvl=1), rec(2, 1, 7, 2), rec(0, 8, 9, 3)], np.uint32)
    L = I.toy_labels(r)
    assert L.complete.tolist() == [17, 20, 2]
    assert L.commit.tolist() == [17, 20, 20]
    assert L.E.tolist() == [17, 20, 2]


def test_mispredicted_branch_redirects_fetch():
    # i0: mispredicted branch, latency 1: issue 1, done 2; next fetch at 2 + 15 = 17
    r = np.array([rec(0, 4, 5, 6, br=1, mp=1), rec(0, 7, 8, 9), rec(0, 10, 11, 12)], np.uint32)
    L = I.toy_labels(r)
    assert L.fetch.tolist() == [0, 17, 17]
    assert L.F.tolist() == [0, 17, 0]
    # a mispredict flag on a non-branch has no effect
    r2 = np.array([rec(0, 4, 5, 6, mp=1), rec(0, 7, 8, 9)], np.uint32)
    assert I.toy_labels(r2).fetch.tolist() == [0, 0]


def test_rob_limits_fetch_and_context_is_in_flight_window():
    # a 200-cycle load at the head blocks commit; instruction 64 waits for it to commit
    r = np.array([rec(0, 30, 31, 1, ld=1, lvl=2)] + [rec(0, 2 + (i % 20), 3, 25) for i in range(70)], np.uint32)
    L = I.toy_labels(r)
    assert L.commit[0] == 1 + 0 + 200 + 1          # issue 1, latency 201
    assert L.fetch[64] == L.commit[0]
    assert (np.diff(L.fetch) >= 0).all() and (np.diff(L.commit) >= 0).all()
    assert (L.commit >= L.complete).all() and (L.complete > L.fetch).all()
    # context of i = uncommitted at fetch[i-1]; contiguous range ending at i-1
    for i in range(1, len(r)):
        j = np.arange(i)
        inflight = j[L.commit[:i] > L.fetch[i - 1]]
        assert L.ctx_begin[i] == (inflight[0] if len(inflight) else i)
        assert (inflight == np.arange(L.ctx_begin[i], i)).all()
