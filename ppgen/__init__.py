"""Seeded synthetic inputs for the peeling workloads.

This module is the one piece shared by the CPU oracle (``oracle/``) and the CUDA
path (``paper_1302_7014_b300``): it only produces inputs -- random keys, random
partitioned hyperedges, the parameters of batched tables and the arrival process
of decode requests.  It holds none of the peeling or hashing arithmetic; the IBLT
cell hashes, checksums and every peeling step are implemented separately on each
side.

Generators (both published, written here from their definitions):

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state_i = seed + i * 0x9E3779B97F4A7C15 and
  output_i = mix(state_i) with the 64-bit finaliser given there.  It is
  counter-based, so any stretch of the stream is computed directly.  Because
  ``mix`` is a bijection of 64-bit words and the increment is odd, the first
  2^64 outputs are pairwise distinct: keys drawn from it are distinct by
  construction.
* xorshift64* (Vigna, "An experimental exploration of Marsaglia's xorshift
  generators, scrambled", ACM TOMS 2016): x ^= x >> 12; x ^= x << 25;
  x ^= x >> 27; output = x * 0x2545F4914F6CDD1D.

The long streams run in the small C helper ``_gen.c`` (compiled with gcc on
first use); the scalar Python forms below are the check on it.

Workload recipes (sizes from the paper's experiments and the stated configs):

* ``PLAIN_PEEL``: r=3, k=2, n=2^14 vertices in 3 parts, m=floor(0.70 n) edges.
* ``IBLT_HEADLINE``: 2^26 cells, r=3, m=0.75*2^26 keys.
* ``DENSITY_SWEEP``: n=2^25, r=4, k=2, c in {0.70,0.76,0.78,0.80,0.85}.
* ``batch_tables``: 4096 IBLTs, cells log-uniform in [2^8, 2^20), r in {3,4},
  c uniform in [0.5, 0.9*c*_{2,r}].
* ``serving_requests``: Poisson arrivals, cells log-uniform in [2^10, 2^22),
  r=3, c uniform in [0.6, 0.8].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15
XS_MULT = 0x2545F4914F6CDD1D

_U64 = np.uint64


# ----------------------------------------------------------------------------
# SplitMix64
# ----------------------------------------------------------------------------
def splitmix64_mix_int(z: int) -> int:
    """SplitMix64 output finaliser on a Python int (scalar)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_first(seed: int) -> int:
    """First output of a SplitMix64 generator whose state starts at ``seed``."""
    return splitmix64_mix_int((seed + SPLITMIX_GAMMA) & MASK64)


def _clib():
    """The compiled stream helper (``_gen.c``), built with gcc on first use."""
    global _CLIB
    if _CLIB is None:
        import ctypes
        import os
        import subprocess
        import tempfile
        here = os.path.dirname(os.path.abspath(__file__))
        src_path = os.path.join(here, "_gen.c")
        so_path = os.path.join(here, "_gen.so")
        if (not os.path.exists(so_path)
                or os.path.getmtime(so_path) < os.path.getmtime(src_path)):
            fd, tmp = tempfile.mkstemp(suffix=".so", dir=here)
            os.close(fd)
            subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src_path])
            os.replace(tmp, so_path)
        lib = ctypes.CDLL(so_path)
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.ppgen_splitmix64.argtypes = [u64, u64, u64, vp]
        lib.ppgen_xorshift64star.argtypes = [u64, u64, vp]
        lib.ppgen_edges.argtypes = [u64, u64, u32, vp, vp, vp]
        _CLIB = lib
    return _CLIB


_CLIB = None


def splitmix64_stream(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 seeded with ``seed``.

    Output i (0-based) is mix(seed + (i+1)*gamma).
    """
    out = np.empty(int(count), dtype=np.uint64)
    if count:
        _clib().ppgen_splitmix64(seed & MASK64, int(start), int(count), out.ctypes.data)
    return out


def distinct_keys(m: int, seed: int) -> np.ndarray:
    """m pairwise-distinct uniform uint64 keys: the first m SplitMix64 outputs."""
    return splitmix64_stream(seed, m)


# ----------------------------------------------------------------------------
# xorshift64*
# ----------------------------------------------------------------------------
def xorshift64star_seed_state(seed: int) -> int:
    """Initial (non-zero) xorshift64 state for a user seed."""
    s = splitmix64_first(seed)
    return s if s != 0 else SPLITMIX_GAMMA


class XorShift64Star:
    """Scalar xorshift64* (reference form, used for small draws and tests)."""

    def __init__(self, seed: int):
        self.state = xorshift64star_seed_state(seed)

    def next(self) -> int:
        x = self.state
        x ^= x >> 12
        x ^= (x << 25) & MASK64
        x ^= x >> 27
        self.state = x
        return (x * XS_MULT) & MASK64

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits of one draw."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def xorshift64star_stream(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of xorshift64* seeded with ``seed``."""
    out = np.empty(int(count), dtype=np.uint64)
    if count:
        _clib().ppgen_xorshift64star(seed & MASK64, int(count), out.ctypes.data)
    return out


def uniform01(draws: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws >> _U64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ----------------------------------------------------------------------------
# Partitioned r-uniform hypergraphs (each edge: one uniform vertex per part)
# ----------------------------------------------------------------------------
def part_sizes(n: int, r: int) -> list[int]:
    """Part j holds floor(n/r) + [j < n mod r] vertices (the paper's parts are
    'equal-sized'; this is the split when r does not divide n)."""
    q, rem = divmod(int(n), int(r))
    return [q + (1 if j < rem else 0) for j in range(r)]


def part_offsets(n: int, r: int) -> list[int]:
    sizes = part_sizes(n, r)
    offs = [0]
    for s in sizes:
        offs.append(offs[-1] + s)
    return offs


def mulhi_u64_u32(u: np.ndarray, s: int) -> np.ndarray:
    """floor(u * s / 2^64) for uint64 u and 0 < s < 2^32 (multiply-shift range map)."""
    assert 0 < s < (1 << 32)
    s64 = _U64(s)
    with np.errstate(over="ignore"):
        hi = u >> _U64(32)
        lo = u & _U64(0xFFFFFFFF)
        return (hi * s64 + ((lo * s64) >> _U64(32))) >> _U64(32)


def edges_from_c(c: float, n: int) -> int:
    """m = floor(c*n) computed in double precision."""
    return int(math.floor(float(c) * float(n)))


def _edges(seed: int, m: int, offs: list[int], sizes: list[int]) -> np.ndarray:
    r = len(sizes)
    out = np.empty((int(m), r), dtype=np.uint32)
    if m:
        o = np.asarray(offs[:r], dtype=np.uint32)
        s = np.asarray(sizes, dtype=np.uint32)
        _clib().ppgen_edges(seed & MASK64, int(m), r, o.ctypes.data, s.ctypes.data,
                            out.ctypes.data)
    return out


def partitioned_edges(n: int, r: int, m: int, seed: int) -> np.ndarray:
    """m edges as an (m, r) uint32 array; endpoint j lies in part j.

    Draw e*r + j of xorshift64*(seed) picks endpoint j of edge e as
    off_j + floor(draw * size_j / 2^64).
    """
    return _edges(seed, m, part_offsets(n, r), part_sizes(n, r))


def uniform_edges(n: int, r: int, m: int, seed: int) -> np.ndarray:
    """m edges with r endpoints each uniform over all n vertices (repeats allowed)."""
    return _edges(seed, m, [0] * r, [int(n)] * r)


# ----------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------
# The paper prints c*_{2,3} ~ 0.818 and c*_{2,4} ~ 0.772 (Section 2); the batch
# recipe uses those printed values so that input generation needs no solver.
CSTAR_PRINTED = {3: 0.818, 4: 0.772}

PLAIN_PEEL = dict(name="plain-peel n=2^14 r=3 k=2 c=0.70", n=1 << 14, r=3, k=2, c=0.70, seed=1)
IBLT_HEADLINE = dict(name="iblt n=2^26 r=3 c=0.75", n_cells=1 << 26, r=3, c=0.75,
                     key_seed=2, table_seed=0x13027014)
DENSITY_SWEEP = dict(name="density-sweep n=2^25 r=4 k=2", n=1 << 25, r=4, k=2,
                     cs=(0.70, 0.76, 0.78, 0.80, 0.85), seed=3)


@dataclass(frozen=True)
class TableSpec:
    """One IBLT of a batch or one decode request."""
    n_cells: int
    r: int
    c: float
    m: int
    table_seed: int   # seed from which each side derives its hash seeds
    key_seed: int     # seed of the SplitMix64 key stream

    def keys(self) -> np.ndarray:
        return distinct_keys(self.m, self.key_seed)


def batch_tables(count: int = 4096, seed_base: int = 4 << 32, lo_log2: int = 8,
                 hi_log2: int = 20, c_lo: float = 0.5, c_frac: float = 0.9,
                 rs: tuple = (3, 4)) -> list[TableSpec]:
    """Tables of the batched workload.

    Table i draws from xorshift64*(splitmix64_first(seed_base + i)):
    u -> cells = floor(2^(lo + (hi-lo) u)), then r = rs[draw & 1], then
    c = c_lo + u' (c_frac * c*_{2,r} - c_lo), m = floor(c * cells).
    """
    out = []
    for i in range(count):
        tseed = splitmix64_first(seed_base + i)
        g = XorShift64Star(tseed)
        u = g.uniform()
        cells = int(math.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)))
        r = rs[g.next() & 1] if len(rs) == 2 else rs[g.next() % len(rs)]
        c = c_lo + g.uniform() * (c_frac * CSTAR_PRINTED[r] - c_lo)
        m = edges_from_c(c, cells)
        out.append(TableSpec(cells, r, c, m, table_seed=tseed,
                             key_seed=splitmix64_first(tseed ^ 0x5BD1E995)))
    return out


def serving_requests(count: int, rate_per_s: float = 20000.0, seed: int = 5,
                     lo_log2: int = 10, hi_log2: int = 22, r: int = 3,
                     c_lo: float = 0.6, c_hi: float = 0.8):
    """(arrival_seconds, TableSpec) for an open-loop Poisson stream of requests."""
    g = XorShift64Star(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log1p(-g.uniform()) / rate_per_s
        u = g.uniform()
        cells = int(math.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)))
        c = c_lo + g.uniform() * (c_hi - c_lo)
        m = edges_from_c(c, cells)
        tseed = splitmix64_first((seed << 40) + i)
        out.append((t, TableSpec(cells, r, c, m, table_seed=tseed,
                                 key_seed=splitmix64_first(tseed ^ 0x5BD1E995))))
    return out


def distinct_uniform_edges(n: int, r: int, m: int, seed: int) -> np.ndarray:
    """m edges of G^r_{n,cn}: r distinct vertices each, uniform (Sec. 2).

    Rows that repeat a vertex are redrawn from further xorshift64* streams
    (seed + 1, seed + 2, ...) until every row is repeat-free."""
    out = uniform_edges(n, r, m, seed)
    bad = np.nonzero(_has_repeat(out))[0]
    bump = 1
    while bad.size:
        out[bad] = uniform_edges(n, r, bad.size, seed + bump)
        bad = bad[_has_repeat(out[bad])]
        bump += 1
    return out


def _has_repeat(rows: np.ndarray) -> np.ndarray:
    """Per row: does some vertex appear twice?"""
    bad = np.zeros(rows.shape[0], dtype=bool)
    for a in range(rows.shape[1]):
        for b in range(a + 1, rows.shape[1]):
            bad |= rows[:, a] == rows[:, b]
    return bad


def trials_union(n: int, r: int, m: int, trials: int, seed: int, kind: str = "distinct"):
    """`trials` independent hypergraphs of n vertices and m edges as one
    hypergraph on trials * n vertices (their disjoint union), so that one peel
    runs every trial at once: trials never share a vertex, so each peels
    exactly as it would alone.

    kind="distinct": G^r_{n,cn} (r distinct vertices per edge); trial i owns
    vertex ids i*n .. (i+1)*n - 1.  kind="partitioned": one vertex per part
    (the sub-table model); the union keeps r contiguous parts, part j holding
    part j of every trial in trial order, so that a sub-round of part j is the
    sub-round of part j in every trial.

    Returns (edges (trials*m, r) uint32, union part offsets (r+1 ints) or None,
    to_trials) where to_trials(x) maps a per-vertex array of the union to a
    (trials, n) array in each trial's own vertex order."""
    T = int(trials)
    if kind == "distinct":
        e = distinct_uniform_edges(n, r, m * T, seed)
        e += (np.arange(T, dtype=np.uint64).repeat(m) * n).astype(np.uint32)[:, None]
        return e, None, lambda x: np.asarray(x).reshape(T, n)
    if kind != "partitioned":
        raise ValueError(kind)
    offs, sizes = part_offsets(n, r), part_sizes(n, r)
    e = _edges(seed, m * T, offs, sizes)
    trial = np.arange(T, dtype=np.int64).repeat(m)
    for j in range(r):
        col = e[:, j].astype(np.int64)
        e[:, j] = (T * offs[j] + trial * sizes[j] + (col - offs[j])).astype(np.uint32)
    uoff = [T * o for o in offs[:r]] + [T * n]

    def to_trials(x):
        x = np.asarray(x)
        return np.concatenate([x[uoff[j]:uoff[j + 1]].reshape(T, sizes[j]) for j in range(r)], axis=1)
    return e, uoff, to_trials
