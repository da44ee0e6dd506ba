"""Brute-force definitions for tiny hypergraphs (pure Python).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  These restate the
definitions with no bookkeeping, to pin the C oracle:

* ``kcore_bruteforce``: the k-core as the largest vertex set whose induced
  sub-hypergraph has minimum degree >= k (Sec. 1: the maximal such subgraph; it
  is unique, so it equals the union of all such sets).
* ``rounds_by_sets``: the round rule of Sec. 1 with sets recomputed from
  scratch every round: remove every vertex of degree < k, and every edge that
  touches one.
* ``subrounds_by_sets``: the sub-table rule of App. B with the same
  from-scratch sets: sub-round j of each round looks at part j only.
"""
from __future__ import annotations


def _degrees(vs, es, edges):
    deg = {v: 0 for v in vs}
    for e in es:
        for u in edges[e]:
            if u in deg:
                deg[u] += 1
    return deg


def kcore_bruteforce(n: int, k: int, edges) -> tuple[frozenset, frozenset]:
    """(core vertices, core edge ids) by enumerating all 2^n vertex subsets."""
    edges = [tuple(int(u) for u in e) for e in edges]
    best = frozenset()
    union = set()
    for mask in range(1 << n):
        s = frozenset(v for v in range(n) if mask >> v & 1)
        inside = [i for i, e in enumerate(edges) if all(u in s for u in e)]
        deg = _degrees(s, inside, edges)
        if all(deg[v] >= k for v in s):
            union |= s
            if len(s) > len(best):
                best = s
    assert frozenset(union) == best, "the maximal set must contain every valid set"
    core_edges = frozenset(i for i, e in enumerate(edges) if all(u in best for u in e))
    return best, core_edges


def rounds_by_sets(n: int, k: int, edges):
    """Returns (vround list, eround list, s_t list, m_t list, T)."""
    edges = [tuple(int(u) for u in e) for e in edges]
    V = set(range(n))
    E = set(range(len(edges)))
    vround = [0] * n
    eround = [0] * len(edges)
    s, m = [], []
    t = 0
    while True:
        deg = _degrees(V, E, edges)
        R = {v for v in V if deg[v] < k}
        if not R:
            break
        t += 1
        D = {e for e in E if any(u in R for u in edges[e])}
        for v in R:
            vround[v] = t
        for e in D:
            eround[e] = t
        V -= R
        E -= D
        s.append(len(V))
        m.append(len(E))
    return vround, eround, s, m, t


def subrounds_by_sets(n: int, k: int, edges, parts):
    """parts: list of vertex-id lists, one per part, visited in order each round.
    Returns (vround, eround, s list, m list, S) with sub-rounds numbered from 1
    and S the last sub-round that removed a vertex."""
    edges = [tuple(int(u) for u in e) for e in edges]
    V = set(range(n))
    E = set(range(len(edges)))
    vround = [0] * n
    eround = [0] * len(edges)
    s, m = [], []
    S = 0
    sub = 0
    idle = 0
    while idle < len(parts):
        part = set(parts[sub % len(parts)])
        sub += 1
        deg = _degrees(V, E, edges)
        R = {v for v in V & part if deg[v] < k}
        if R:
            idle = 0
            S = sub
        else:
            idle += 1
        D = {e for e in E if any(u in R for u in edges[e])}
        for v in R:
            vround[v] = sub
        for e in D:
            eround[e] = sub
        V -= R
        E -= D
        s.append(len(V))
        m.append(len(E))
    return vround, eround, s[:S], m[:S], S
