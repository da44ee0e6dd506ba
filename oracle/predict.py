"""Idealised predictions for parallel peeling (fp64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``cstar``: the threshold c*_{k,r} of Eq. 2.1 (Sec. 2), minimised over x > 0.
* ``recurrence``: rho_i, beta_i, lambda_i of Sec. 3.1 (Eqs. 3.1-3.4): a vertex
  survives i rounds with probability lambda_i, a vertex hanging off an edge of
  the branching tree with probability rho_i.  An edge survives i rounds iff all
  r of its endpoints do, which gives the expected surviving-edge fraction
  rho_i^r.
* ``fixed_point``: the above-threshold limit beta of Eq. 4.1 (Sec. 4), with
  lambda (core vertex fraction), rho and the core edge fraction rho^r.
* ``subtable_recurrence``: rho_{i,j}, lambda_{i,j} and lambda'_{i,j} of App. B
  (peeling with r sub-tables, one sub-table per sub-round).

The Poisson tail P(Poi(mu) >= k) is evaluated as a forward series when mu is
small (no cancellation), else as one minus the head.
"""
from __future__ import annotations

import math


def poisson_sf(k: int, mu: float) -> float:
    """P(Poisson(mu) >= k)."""
    if k <= 0:
        return 1.0
    if mu <= 0.0:
        return 0.0
    if mu < k + 1.0:
        term = math.exp(-mu + k * math.log(mu) - math.lgamma(k + 1))
        s, j = 0.0, k
        while term > 0.0 and (term > s * 1e-18) and j < k + 10000:
            s += term
            j += 1
            term *= mu / j
        return s
    head, term = 0.0, math.exp(-mu)
    for j in range(k):
        head += term
        term *= mu / (j + 1)
    return 1.0 - head


def _cstar_objective(x: float, k: int, r: int) -> float:
    p = poisson_sf(k - 1, x)   # 1 - e^{-x} sum_{j<=k-2} x^j/j!
    if p <= 0.0:
        return math.inf
    return x / (r * p ** (r - 1))


def cstar(k: int, r: int) -> tuple[float, float]:
    """(c*_{k,r}, argmin x*) from Eq. 2.1: min_{x>0} x / (r (P(Poi(x) >= k-1))^{r-1})."""
    if k == 2 and r == 2:
        raise ValueError("k = r = 2 is excluded (Sec. 2)")
    xs = [10 ** (-3 + 5 * i / 4000) for i in range(4001)]
    vals = [_cstar_objective(x, k, r) for x in xs]
    i = min(range(len(xs)), key=vals.__getitem__)
    lo, hi = xs[max(0, i - 1)], xs[min(len(xs) - 1, i + 1)]
    g = (math.sqrt(5) - 1) / 2
    a, b = lo, hi
    c1, c2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = _cstar_objective(c1, k, r), _cstar_objective(c2, k, r)
    for _ in range(200):
        if f1 < f2:
            b, c2, f2 = c2, c1, f1
            c1 = b - g * (b - a)
            f1 = _cstar_objective(c1, k, r)
        else:
            a, c1, f1 = c1, c2, f2
            c2 = a + g * (b - a)
            f2 = _cstar_objective(c2, k, r)
    x = 0.5 * (a + b)
    return _cstar_objective(x, k, r), x


def recurrence(k: int, r: int, c: float, rounds: int):
    """Lists beta[1..T], rho[0..T], lam[1..T] of Sec. 3.1 (index 0 of beta/lam unused)."""
    rho = [1.0]
    beta = [math.nan]
    lam = [1.0]
    for _ in range(rounds):
        b = rho[-1] ** (r - 1) * r * c
        beta.append(b)
        rho.append(poisson_sf(k - 1, b))
        lam.append(poisson_sf(k, b))
    return beta, rho, lam


def expected_vertices(n: int, k: int, r: int, c: float, rounds: int) -> list[float]:
    """n * lambda_t for t = 1..rounds (the 'Prediction' column of Table 2)."""
    _, _, lam = recurrence(k, r, c, rounds)
    return [n * x for x in lam[1:]]


def expected_edges(m: int, k: int, r: int, c: float, rounds: int) -> list[float]:
    """m * rho_t^r for t = 1..rounds: expected edges (IBLT keys) left after t rounds."""
    _, rho, _ = recurrence(k, r, c, rounds)
    return [m * x ** r for x in rho[1:]]


def predicted_rounds(n: int, k: int, r: int, c: float, limit: int = 10000) -> int:
    """First t with n * lambda_t < 1 (rounds to an empty core in the idealised model)."""
    _, _, lam = recurrence(k, r, c, limit)
    for t in range(1, limit + 1):
        if n * lam[t] < 1.0:
            return t
    return limit


def fixed_point(k: int, r: int, c: float, iters: int = 100000, tol: float = 1e-15):
    """Above-threshold limit of beta_i (Eq. 4.1).  Returns dict(beta, rho, lam, edge_frac)."""
    b = r * c
    for _ in range(iters):
        nb = poisson_sf(k - 1, b) ** (r - 1) * r * c
        if abs(nb - b) <= tol * max(1.0, b):
            b = nb
            break
        b = nb
    rho = poisson_sf(k - 1, b)
    return dict(beta=b, rho=rho, lam=poisson_sf(k, b), edge_frac=rho ** r)


def fprime0(k: int, r: int, beta: float) -> float:
    """f'(0) of Eq. 4.3 at the fixed point beta (0 < f'(0) < 1 above threshold)."""
    p = poisson_sf(k - 1, beta)
    return (r - 1) * beta * math.exp(-beta) / p * beta ** (k - 2) / math.factorial(k - 2)


def subtable_recurrence(k: int, r: int, c: float, rounds: int):
    """App. B: returns (rho, lam, lam_prime) with rho[i][j], lam[i][j] for
    i = 0..rounds, j = 0..r-1 (sub-table j+1 of the paper), and lam_prime[i][j]
    for i >= 1 = the expected fraction of vertices left after sub-round (i, j+1)."""
    rho = [[1.0] * r]
    lam = [[1.0] * r]
    for i in range(1, rounds + 1):
        rho_i, lam_i = [0.0] * r, [0.0] * r
        for j in range(r):
            b = r * c
            for h in range(j):
                b *= rho_i[h]
            for h in range(j + 1, r):
                b *= rho[i - 1][h]
            rho_i[j] = poisson_sf(k - 1, b)
            lam_i[j] = poisson_sf(k, b)
        rho.append(rho_i)
        lam.append(lam_i)
    lam_prime = [[math.nan] * r]
    for i in range(1, rounds + 1):
        row = []
        for j in range(r):
            s = sum(lam[i][h] for h in range(j + 1)) + sum(lam[i - 1][h] for h in range(j + 1, r))
            row.append(s / r)
        lam_prime.append(row)
    return rho, lam, lam_prime


def fibonacci_growth(order: int) -> float:
    """Growth rate of the order-`order` Fibonacci sequence (each term the sum of
    the previous `order` terms): the root in (1, 2) of x^o = x^{o-1} + ... + 1."""
    lo, hi = 1.0, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid ** order - sum(mid ** i for i in range(order)) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def loglog_rounds_term(n: int, k: int, r: int) -> float:
    """log log n / log((k-1)(r-1)): the n-dependent part of Theorems 1 and 2."""
    return math.log(math.log(n)) / math.log((k - 1) * (r - 1))
