"""Statistical pins: the oracle's round simulator against the paper's simulations.

Table 1 gives mean rounds over 1000 hypergraphs G^r_{n,cn} (r distinct
vertices per edge), r = 4, k = 2.  We draw fewer hypergraphs and accept a
difference of 4 standard errors of our own mean (plus 0.02 for the paper's
rounding).  These pin what a "round" is: a reading that also counted the final
no-change round would sit a full round above the table.
"""
import math

import numpy as np
import pytest

import oracle
import ppgen
from conftest import read_golden
from oracle import predict as P


def _rounds(n, c, trials, seed0, r=4, k=2):
    m = ppgen.edges_from_c(c, n)
    out, fails = [], 0
    for t in range(trials):
        e = ppgen.distinct_uniform_edges(n, r, m, seed0 + 7919 * t)
        res = oracle.kcore_rounds(n, k, e)
        out.append(res["rounds"])
        fails += int(res["s"][-1] > 0) if res["s"] else 0
    return np.array(out, float), fails


@pytest.mark.parametrize("col,c", [(1, 0.70), (3, 0.75), (5, 0.80), (7, 0.85)])
def test_table1_mean_rounds_n1e4(col, c):
    row = read_golden("table1_rounds.txt")[0]
    assert int(row[0]) == 10000
    want_fail, want_rounds = int(row[col]), float(row[col + 1])
    rounds, fails = _rounds(10000, c, 300, 1000 + int(100 * c))
    se = rounds.std(ddof=1) / math.sqrt(rounds.size)
    assert abs(rounds.mean() - want_rounds) < 4 * se + 0.02
    # all trials fail above c*_{2,4} ~ 0.772 and none below (Table 1)
    assert fails == (300 if want_fail == 1000 else 0)


@pytest.mark.slow
def test_table2_survivors_one_hypergraph():
    # one G^4_{n,0.7n} with n = 10^6 against Table 2's experiment column (a
    # mean over 1000 draws).  The cascade makes later rounds of one draw vary by
    # a few thousand vertices; the first round varies by ~sqrt(n).
    rows = read_golden("table2_prediction.txt")
    e = ppgen.distinct_uniform_edges(10**6, 4, 700000, 17)
    res = oracle.kcore_rounds(10**6, 2, e)
    s = res["s"] + [0] * 20
    assert abs(s[0] - float(rows[0][2])) < 5 * math.sqrt(10**6 * 0.77 * 0.23)
    for row in rows[:11]:
        t, exp = int(row[0]), float(row[2])
        assert abs(s[t - 1] - exp) < 5000, t
    assert abs(s[11] - float(rows[11][2])) < 60
    assert s[12] == 0 and res["rounds"] == 13


def test_partitioned_first_round_matches_prediction():
    # the partitioned hypergraph has the same Poisson(rc) degrees: n lambda_1
    # predicts the survivors after round 1 of the r = 4, c = 0.7 draw
    n = 400000
    e = ppgen.partitioned_edges(n, 4, ppgen.edges_from_c(0.7, n), 5)
    res = oracle.kcore_rounds(n, 2, e)
    pred = P.expected_vertices(n, 2, 4, 0.7, 3)
    for t in range(3):
        assert abs(res["s"][t] - pred[t]) < 6 * math.sqrt(n), t


def test_loglog_below_threshold_and_log_above():
    # Theorems 1-3: below c* rounds barely move with n; above c* they grow ~ log n
    below = [_rounds(n, 0.70, 40, 50)[0].mean() for n in (10000, 160000)]
    above = [_rounds(n, 0.85, 40, 60)[0].mean() for n in (10000, 160000)]
    assert below[1] - below[0] < 1.0
    # Table 1 at c = 0.85: 10.773 -> 15.005 over the same range of n
    assert 2.5 < above[1] - above[0] < 6.0
