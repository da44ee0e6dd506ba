"""The idealised predictors against the values the paper prints."""
import math

import pytest

from conftest import read_golden
from oracle import predict as P


def _constants(kind):
    return [r[1:] for r in read_golden("printed_constants.txt") if r[0] == kind]


@pytest.mark.parametrize("row", _constants("cstar"), ids=lambda r: f"c*_{r[0]},{r[1]}")
def test_cstar_printed(row):
    k, r, value, digits = int(row[0]), int(row[1]), float(row[2]), int(row[3])
    c, x = P.cstar(k, r)
    assert round(c, digits) == pytest.approx(value, abs=1e-12)
    # x* is a minimiser: the objective is larger on both sides
    assert P._cstar_objective(x * 0.99, k, r) > c and P._cstar_objective(x * 1.01, k, r) > c


def test_cstar_closed_form_k2():
    # at k = 2 the objective is x / (r (1 - e^-x)^(r-1)); its stationary point
    # solves (1 - e^-x) = (r - 1) x e^-x
    for r in (3, 4, 5, 6):
        c, x = P.cstar(2, r)
        assert abs((1 - math.exp(-x)) - (r - 1) * x * math.exp(-x)) < 1e-6
        assert abs(c - x / (r * (1 - math.exp(-x)) ** (r - 1))) < 1e-12


def test_table2_prediction_columns():
    rows = read_golden("table2_prediction.txt")
    p07 = P.expected_vertices(10**6, 2, 4, 0.70, len(rows))
    p085 = P.expected_vertices(10**6, 2, 4, 0.85, len(rows))
    for row, a, b in zip(rows, p07, p085):
        t = int(row[0])
        if "." in row[1]:                     # printed with 5 decimals
            assert round(a, 5) == float(row[1]), t
        else:
            assert round(a) == int(row[1]), t
        assert round(b) == int(row[3]), t


def test_table6_prediction_column():
    rows = read_golden("table6_prediction.txt")
    _, _, lp = P.subtable_recurrence(2, 4, 0.70, 7)
    for row in rows:
        i, j, want = int(row[0]), int(row[1]), row[2]
        got = 10**6 * lp[i][j - 1]
        if "." in want:
            assert round(got, 3) == float(want), (i, j)
        else:
            assert round(got) == int(want), (i, j)


def test_first_round_closed_form():
    # lambda_1 = P(Poi(rc) >= k): every vertex with initial degree >= k survives round 1
    for k, r, c in ((2, 4, 0.7), (2, 3, 0.75), (3, 3, 1.2)):
        _, _, lam = P.recurrence(k, r, c, 1)
        mu = r * c
        head = sum(math.exp(-mu) * mu**j / math.factorial(j) for j in range(k))
        assert abs(lam[1] - (1 - head)) < 1e-15


def test_poisson_tail_branches_agree():
    for k in range(0, 6):
        for mu in (1e-6, 0.01, 0.5, 1.0, 2.8, 5.0, 7.5, 30.0):
            direct = 1 - sum(math.exp(-mu) * mu**j / math.factorial(j) for j in range(k))
            assert abs(P.poisson_sf(k, mu) - direct) < 1e-12


@pytest.mark.parametrize("row", _constants("fib"), ids=lambda r: f"fib{r[0]}")
def test_fibonacci_growth_printed(row):
    order, value, digits = int(row[0]), float(row[1]), int(row[2])
    phi = P.fibonacci_growth(order)
    assert math.floor(phi * 10**digits) / 10**digits == pytest.approx(value)


def test_subtable_ratio_printed():
    # App. B prints log(r-1)/log(phi_{r-1}) ~ 1.456 for r = 3; that figure is
    # what phi rounded to the printed 1.61 gives (1.4555).  With the exact golden
    # ratio the ratio is 1.440, still "less than 1.5" as the paper states.
    row = _constants("ratio")[0]
    r = int(row[0])
    assert abs(math.log(r - 1) / math.log(1.61) - float(row[1])) < 1e-3
    exact = math.log(r - 1) / math.log(P.fibonacci_growth(r - 1))
    assert abs(exact - 1.4404) < 1e-4 and exact < 1.5


def test_above_threshold_recovered_fraction_r4():
    # Table 4: 24.6 % recovered at load 0.83, r = 4 (2^24 cells).  Keys left in
    # the core ~ m rho^r, so the recovered share is 1 - rho^r.
    rec = dict(((int(r[0]), float(r[1])), float(r[2])) for r in _constants("recovered"))
    fp = P.fixed_point(2, 4, 0.83)
    assert abs(100 * (1 - fp["edge_frac"]) - rec[(4, 0.83)]) < 0.05
    # r = 3: the asymptotic value (52.3 %) sits 2.2 points above the printed
    # 50.1 %; the gap is not explained in the paper, so only a loose bound.
    fp3 = P.fixed_point(2, 3, 0.83)
    assert abs(100 * (1 - fp3["edge_frac"]) - rec[(3, 0.83)]) < 3.0


def test_fixed_point_slope_in_unit_interval():
    # Eq. 4.4: 0 < f'(0) < 1 above the threshold
    for k, r, c in ((2, 4, 0.8), (2, 3, 0.85), (3, 3, 1.7)):
        fp = P.fixed_point(k, r, c)
        assert fp["beta"] > 0
        assert 0 < P.fprime0(k, r, fp["beta"]) < 1
    # below the threshold the limit is beta = 0
    assert P.fixed_point(2, 4, 0.7)["beta"] < 1e-12


def test_doubly_exponential_decay_below_threshold():
    # Sec. 3.1: once beta is small, beta_{i+1} <= beta_i^{(k-1)(r-1)} rc/[(k-1)!]^{r-1}
    for k, r, c in ((2, 4, 0.7), (2, 3, 0.75), (3, 3, 1.4)):
        beta, _, _ = P.recurrence(k, r, c, 40)
        bound = r * c / math.factorial(k - 1) ** (r - 1)
        for i in range(1, 39):
            if 0 < beta[i] < 0.05 and beta[i + 1] > 0:
                assert beta[i + 1] <= beta[i] ** ((k - 1) * (r - 1)) * bound * (1 + 1e-9)
