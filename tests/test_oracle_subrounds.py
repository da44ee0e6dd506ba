"""Pins for the sub-table (sub-round) peel of App. B in the oracle.

App. B: the vertices are split into r parts and each round runs one
sub-round per part; a sub-round removes the vertices of its part whose degree
is < k at that moment.  These tests pin the oracle's ``kcore_subrounds`` and
``IBLT.decode_subrounds`` against things other than themselves:

* a hand-worked example;
* the from-scratch set simulation of ``oracle/brute.py`` on tiny hypergraphs;
* the special case of one part, which is the round process of Sec. 1;
* the k-core itself (unique, Sec. 1), which every peeling order reaches;
* Table 5 (mean sub-rounds at n = 10^4) and Table 6 (vertices left after
  each sub-round at n = 10^6), statistically;
* for the IBLT, the k = 2 sub-round peel of the key hypergraph.
"""
import math

import numpy as np
import pytest

import oracle
import ppgen
from conftest import read_golden
from oracle import brute


def _offsets(n, p):
    return [int(x) for x in oracle.part_offsets(n, p)]


def _rand_hypergraph(rng, n, r, m):
    return rng.integers(0, n, size=(m, r), dtype=np.uint32)


def test_hand_worked_path():
    # the path 0 - 2 - 1 - 3 (edges (0,2), (2,1), (1,3); r = 2, k = 2) with
    # part 0 = {0, 1} and part 1 = {2, 3}.
    # Sub-round 1 (part 0): deg(0) = 1 -> 0 goes, with (0,2).
    # Sub-round 2 (part 1): deg(2) = 1, deg(3) = 1 -> both go, with (2,1) and
    # (1,3).  Sub-round 3 (part 0): deg(1) = 0 -> 1 goes.  Two idle sub-rounds
    # follow, so S = 3.
    e = np.array([[0, 2], [2, 1], [1, 3]], dtype=np.uint32)
    res = oracle.kcore_subrounds(4, 2, e, [0, 2, 4])
    assert res["subrounds"] == 3
    assert list(res["vround"]) == [1, 3, 2, 2]
    assert list(res["eround"]) == [1, 2, 2]
    assert res["s"] == [3, 1, 0]
    assert res["m"] == [2, 0, 0]
    # the full-round process needs 2 rounds on the same path
    assert oracle.kcore_rounds(4, 2, e)["rounds"] == 2


def test_hand_worked_idle_part_in_the_middle():
    # part 1 has nothing to remove in round 1, part 2 does: the idle sub-round
    # keeps its number and its counts.  Edges: (0,1,4) and (2,3,4), k = 2;
    # vertex 4 (part 2) has degree 2, every other vertex degree 1.  Parts:
    # {0,1} {} {2,3,4}.
    e = np.array([[0, 1, 4], [2, 3, 4]], dtype=np.uint32)
    res = oracle.kcore_subrounds(5, 2, e, [0, 2, 2, 5])
    # sub-round 1: 0 and 1 go with edge 0 -> deg(4) = 1
    # sub-round 2: part 1 is empty (idle)
    # sub-round 3: 2, 3, 4 go with edge 1
    assert res["subrounds"] == 3
    assert list(res["vround"]) == [1, 1, 3, 3, 3]
    assert list(res["eround"]) == [1, 3]
    assert res["s"] == [3, 3, 0]
    assert res["m"] == [1, 1, 0]


def test_one_part_is_the_round_process():
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(1, 300))
        r = int(rng.integers(1, 5))
        m = int(rng.integers(0, 2 * n))
        k = int(rng.integers(1, 4))
        e = _rand_hypergraph(rng, n, r, m)
        a = oracle.kcore_rounds(n, k, e)
        b = oracle.kcore_subrounds(n, k, e, [0, n])
        assert b["subrounds"] == a["rounds"], trial
        assert np.array_equal(a["vround"], b["vround"]), trial
        assert np.array_equal(a["eround"], b["eround"]), trial
        assert a["s"] == b["s"] and a["m"] == b["m"], trial


def test_tiny_hypergraphs_vs_sets():
    rng = np.random.default_rng(5)
    for trial in range(150):
        n = int(rng.integers(1, 13))
        r = int(rng.integers(1, 5))
        m = int(rng.integers(0, 3 * n))
        k = int(rng.integers(1, 4))
        p = int(rng.integers(1, 5))
        cuts = sorted(int(x) for x in rng.integers(0, n + 1, size=p - 1))
        off = [0] + cuts + [n]
        e = _rand_hypergraph(rng, n, r, m)
        got = oracle.kcore_subrounds(n, k, e, off)
        parts = [list(range(off[j], off[j + 1])) for j in range(p)]
        vr, er, s, mm, S = brute.subrounds_by_sets(n, k, e.tolist(), parts)
        assert got["subrounds"] == S, trial
        assert list(got["vround"]) == vr, trial
        assert list(got["eround"]) == er, trial
        assert got["s"] == s and got["m"] == mm, trial


@pytest.mark.parametrize("k", [2, 3])
def test_reaches_the_k_core(k):
    rng = np.random.default_rng(100 + k)
    for trial in range(10):
        n, r = 3000, int(rng.integers(2, 5))
        m = int(n * (0.6 + 0.3 * rng.random()) * (1 if k == 2 else 2))
        e = ppgen.partitioned_edges(n, r, m, 1000 * k + trial)
        res = oracle.kcore_subrounds(n, k, e, _offsets(n, r))
        vc, ec = oracle.kcore_queue(n, k, e)
        assert np.array_equal(res["vround"] == 0, vc.astype(bool)), trial
        assert np.array_equal(res["eround"] == 0, ec.astype(bool)), trial


def test_no_more_subrounds_than_r_times_rounds():
    # App. B: a round of r sub-rounds removes at least what one full round does
    for seed in range(10):
        n, r = 8000, 4
        e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(0.72, n), 300 + seed)
        a = oracle.kcore_rounds(n, 2, e)
        b = oracle.kcore_subrounds(n, 2, e, _offsets(n, r))
        assert b["subrounds"] <= r * a["rounds"]
        # after round i (sub-round r*i) no more vertices are left than after
        # full round i
        for i in range(1, a["rounds"] + 1):
            left_sub = b["s"][r * i - 1] if r * i <= b["subrounds"] else b["s"][-1]
            assert left_sub <= a["s"][i - 1], (seed, i)


@pytest.mark.parametrize("col,c", [(1, 0.70), (3, 0.75)])
def test_table5_mean_subrounds_n1e4(col, c):
    row = read_golden("table5_subrounds.txt")[0]
    assert int(row[0]) == 10000
    want_fail, want = int(row[col]), float(row[col + 1])
    n, r, trials = 10000, 4, 600
    off = _offsets(n, r)
    m = ppgen.edges_from_c(c, n)
    got, fails = [], 0
    for t in range(trials):
        e = ppgen.partitioned_edges(n, r, m, 5000 + 7919 * t + int(100 * c))
        res = oracle.kcore_subrounds(n, 2, e, off)
        got.append(res["subrounds"])
        fails += int(res["s"][-1] > 0) if res["s"] else 0
    got = np.array(got, float)
    se = got.std(ddof=1) / math.sqrt(trials)
    assert abs(got.mean() - want) < 4 * se + 0.02
    assert fails == want_fail


def test_table6_experiment_column():
    # a few draws of the n = 10^6, r = 4, c = 0.7 partitioned hypergraph
    # against the experiment column (a mean over 1000 draws): within 5
    # standard errors of our own mean, plus the table's rounding
    rows = read_golden("table6_prediction.txt")
    n, r, trials = 10**6, 4, 6
    off = _offsets(n, r)
    runs = []
    for t in range(trials):
        e = ppgen.partitioned_edges(n, r, 700000, 90 + t)
        res = oracle.kcore_subrounds(n, 2, e, off)
        runs.append(res["s"] + [0] * (len(rows) - len(res["s"])))
    a = np.array(runs, float)
    mean = a.mean(0)
    se = a.std(0, ddof=1) / math.sqrt(trials)
    for row in rows:
        i, j, exp = int(row[0]), int(row[1]), float(row[3])
        s = (i - 1) * r + j
        assert abs(mean[s - 1] - exp) < 5 * se[s - 1] + 1.0, (i, j, mean[s - 1], exp)


# ----------------------------------------------------------------------------
# IBLT recovery with sub-tables
# ----------------------------------------------------------------------------
def _iblt(n, r, m, seed, key_seed):
    keys = ppgen.distinct_keys(m, key_seed)
    t = oracle.IBLT(n, r, seed)
    t.insert(keys)
    return t, keys


@pytest.mark.parametrize("n,r,c,seed", [(2000, 3, 0.75, 1), (4096, 4, 0.70, 2), (3001, 3, 0.85, 3),
                                        (1000, 5, 0.6, 4)])
def test_iblt_subrounds_equal_kcore_subrounds(n, r, c, seed):
    m = ppgen.edges_from_c(c, n)
    t, keys = _iblt(n, r, m, seed, 40 + seed)
    cells = oracle.key_cells(n, r, seed, keys).astype(np.uint32)
    ref = oracle.kcore_subrounds(n, 2, cells, _offsets(n, r))
    got = t.decode_subrounds()
    assert got["status"] == oracle.OK
    assert got["subrounds"] == max([0] + [int(x) for x in ref["eround"]])
    for s in range(1, got["subrounds"] + 1):
        want = np.sort(keys[ref["eround"] == s])
        assert np.array_equal(got["keys"][s - 1], want), s


def test_iblt_subrounds_same_outcome_as_rounds():
    # the 2-core is unique: both orders recover the same keys and leave the same
    # residue
    for seed, c in [(7, 0.7), (8, 0.82), (9, 0.9)]:
        n, r = 5000, 3
        t, keys = _iblt(n, r, ppgen.edges_from_c(c, n), seed, seed)
        u = t.copy()
        a = t.decode_rounds()
        b = u.decode_subrounds()
        ka = np.sort(np.concatenate(a["keys"])) if a["keys"] else np.zeros(0, np.uint64)
        kb = np.sort(np.concatenate(b["keys"])) if b["keys"] else np.zeros(0, np.uint64)
        assert np.array_equal(ka, kb)
        assert np.array_equal(t.count, u.count)
        assert np.array_equal(t.keyx, u.keyx) and np.array_equal(t.chkx, u.chkx)


def test_iblt_subrounds_recover_inserted_set_below_threshold():
    n, r = 30000, 3
    t, keys = _iblt(n, r, ppgen.edges_from_c(0.75, n), 12, 13)
    res = t.decode_subrounds()
    got = np.sort(np.concatenate(res["keys"]))
    assert np.array_equal(got, np.sort(keys))
    assert t.residual_cells() == 0
    # no key comes out twice: sub-tables make each key's cells distinct
    assert np.unique(got).size == got.size


def test_iblt_subrounds_empty_table_and_limit():
    t = oracle.IBLT(300, 3, 1)
    res = t.decode_subrounds()
    assert res["subrounds"] == 0 and res["keys"] == [] and res["status"] == oracle.OK
    t, _ = _iblt(3000, 3, 2000, 5, 6)
    res = t.decode_subrounds(max_subrounds=2)
    assert res["status"] == oracle.ROUND_LIMIT
