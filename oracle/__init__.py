"""CPU oracle for round-synchronous parallel peeling.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
``bench.py`` use this package to check the CUDA path.  The library itself never
imports it, and it shares no code with the CUDA path; both sides only share the
seeded input generators in ``ppgen``.

* ``peel_oracle.c`` (compiled with gcc on first use): IBLT insertion,
  round-synchronous and sequential IBLT recovery, round-synchronous and
  sequential k-core peeling, and the sub-table (sub-round) variants of the
  round-synchronous peel and recovery (App. B).
* ``predict.py``: the threshold c*_{k,r} (Eq. 2.1), the idealised recurrences
  for rho_i, lambda_i, beta_i (Sec. 3.1), the above-threshold fixed point
  (Sec. 4) and the sub-table recurrences (App. B).
* ``brute.py``: brute-force k-core and a set-by-set round simulator for tiny
  hypergraphs (pins for the C code).

Parity unpinned: the IBLT cell map and the split of n cells into r
sub-tables are conventions the paper leaves open (Sec. 6 asks for r hash
functions and a pseudorandom checksum without fixing them).  They are fixed
in ``peel_oracle.c`` and frozen by the known-answer file
``tests/golden/hash_kat.txt``, which the CUDA side must reproduce.  The mix64
finaliser inside them is pinned to a published vector, and the range map to
the edges of its equal-width intervals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "peel_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

OK, CAPACITY, ROUND_LIMIT, INVALID, NOMEM = 0, 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile ``peel_oracle.c`` into ``_build/liboracle.so`` (plain -O2, no tuning)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
        os.close(fd)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def configure(so):
    """Declare the C signatures on a loaded copy of the oracle library."""
    if True:
        u64, u32, i64, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
        so.orc_mix64.argtypes = [u64]
        so.orc_mix64.restype = u64
        so.orc_hash_seeds.argtypes = [u64, u32, vp]
        so.orc_part_offsets.argtypes = [u64, u32, vp]
        so.orc_key_cells.argtypes = [u64, u32, u64, vp, u64, vp]
        so.orc_checksum.argtypes = [u64, u32, u64]
        so.orc_checksum.restype = u64
        so.orc_iblt_insert.argtypes = [u64, u32, u64, vp, u64, i64, vp, vp, vp]
        so.orc_iblt_decode_rounds.argtypes = [u64, u32, u64, vp, vp, vp, u32, vp, u64, vp, vp, vp]
        so.orc_iblt_decode_queue.argtypes = [u64, u32, u64, vp, vp, vp, vp, u64, vp]
        so.orc_kcore_rounds.argtypes = [u32, u32, u32, vp, u64, u32, vp, vp, vp, vp, vp]
        so.orc_kcore_queue.argtypes = [u32, u32, u32, vp, u64, vp, vp]
        so.orc_kcore_subrounds.argtypes = [u32, u32, u32, vp, u64, u32, vp, u32, vp, vp, vp, vp, vp]
        so.orc_iblt_decode_subrounds.argtypes = [u64, u32, u64, vp, vp, vp, u32, vp, u64, vp, vp]
        so.orc_iblt_decode_signed.argtypes = [u64, u32, u64, vp, vp, vp, u32, vp, vp, u64, vp, vp]
        for f in ("orc_iblt_insert", "orc_iblt_decode_rounds", "orc_iblt_decode_queue",
                  "orc_kcore_rounds", "orc_kcore_queue", "orc_kcore_subrounds",
                  "orc_iblt_decode_subrounds", "orc_iblt_decode_signed"):
            getattr(so, f).restype = ctypes.c_int
    return so


def lib():
    global _lib
    if _lib is None:
        _lib = configure(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data


# ----------------------------------------------------------------------------
# IBLT
# ----------------------------------------------------------------------------
def mix64(x: int) -> int:
    return int(lib().orc_mix64(x & ((1 << 64) - 1)))


def hash_seeds(table_seed: int, r: int) -> np.ndarray:
    out = np.zeros(r + 1, dtype=np.uint64)
    lib().orc_hash_seeds(table_seed, r, _ptr(out))
    return out


def part_offsets(n: int, r: int) -> np.ndarray:
    out = np.zeros(r + 1, dtype=np.uint64)
    lib().orc_part_offsets(n, r, _ptr(out))
    return out


def key_cells(n: int, r: int, table_seed: int, keys: np.ndarray) -> np.ndarray:
    """(m, r) uint64: the r cells of each key."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.zeros((keys.size, r), dtype=np.uint64)
    lib().orc_key_cells(n, r, table_seed, _ptr(keys), keys.size, _ptr(out))
    return out


def checksum(table_seed: int, r: int, x: int) -> int:
    """checkSum(x) = mix64(x ^ checksum seed), 64 bits."""
    return int(lib().orc_checksum(table_seed, r, x))


class IBLT:
    """A CPU IBLT: per cell the count (int64), the XOR of its keys (uint64) and
    the XOR of their 64-bit checksums (uint64), as Sec. 6 "Motivation" defines
    the cell's fields."""

    def __init__(self, n_cells: int, r: int, table_seed: int):
        self.n, self.r, self.seed = int(n_cells), int(r), int(table_seed)
        self.count = np.zeros(self.n, dtype=np.int64)
        self.keyx = np.zeros(self.n, dtype=np.uint64)
        self.chkx = np.zeros(self.n, dtype=np.uint64)

    def copy(self) -> "IBLT":
        t = IBLT.__new__(IBLT)
        t.n, t.r, t.seed = self.n, self.r, self.seed
        t.count, t.keyx, t.chkx = self.count.copy(), self.keyx.copy(), self.chkx.copy()
        return t

    def insert(self, keys: np.ndarray, sign: int = 1) -> None:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        st = lib().orc_iblt_insert(self.n, self.r, self.seed, _ptr(keys), keys.size, sign,
                                   _ptr(self.count), _ptr(self.keyx), _ptr(self.chkx))
        if st != OK:
            raise ValueError(f"orc_iblt_insert status {st}")

    def decode_rounds(self, max_rounds: int = 1 << 20):
        """Round-synchronous recovery; mutates the table (leaves the 2-core residue).

        Returns dict(keys=[array per round, sorted], rounds=T, cells_alive=[s_1..s_T],
        status=code)."""
        cap = int(max(1, (np.abs(self.count).sum() // self.r) + 1))
        cap = max(cap, self.n)
        out = np.zeros(cap, dtype=np.uint64)
        mr = min(max_rounds, self.n + 2)
        round_end = np.zeros(mr + 1, dtype=np.uint64)
        alive = np.zeros(mr + 1, dtype=np.uint64)
        T = np.zeros(1, dtype=np.uint32)
        st = lib().orc_iblt_decode_rounds(self.n, self.r, self.seed, _ptr(self.count),
                                          _ptr(self.keyx), _ptr(self.chkx), mr, _ptr(out), cap,
                                          _ptr(round_end), _ptr(alive), _ptr(T))
        T = int(T[0])
        ends = [0] + [int(x) for x in round_end[:T]]
        keys = [out[ends[i]:ends[i + 1]].copy() for i in range(T)]
        return dict(keys=keys, rounds=T, cells_alive=[int(x) for x in alive[:T]], status=st)

    def decode_queue(self):
        """Sequential recovery; returns (recovered keys in the order found, status)."""
        cap = max(1, self.n)
        out = np.zeros(cap, dtype=np.uint64)
        got = np.zeros(1, dtype=np.uint64)
        st = lib().orc_iblt_decode_queue(self.n, self.r, self.seed, _ptr(self.count),
                                         _ptr(self.keyx), _ptr(self.chkx), _ptr(out), cap,
                                         _ptr(got))
        return out[: int(got[0])].copy(), st

    def decode_subrounds(self, max_subrounds: int = 1 << 20):
        """Recovery with sub-tables (App. B): one sub-table per sub-round; mutates
        the table.  Returns dict(keys=[array per sub-round, sorted], subrounds=S,
        status=code)."""
        cap = int(max(1, (np.abs(self.count).sum() // self.r) + 1))
        cap = max(cap, self.n)
        out = np.zeros(cap, dtype=np.uint64)
        ms = int(min(max_subrounds, self.r * (self.n + 2)))
        sub_end = np.zeros(ms + 1, dtype=np.uint64)
        S = np.zeros(1, dtype=np.uint32)
        st = lib().orc_iblt_decode_subrounds(self.n, self.r, self.seed, _ptr(self.count),
                                             _ptr(self.keyx), _ptr(self.chkx), ms, _ptr(out), cap,
                                             _ptr(sub_end), _ptr(S))
        S = int(S[0])
        ends = [0] + [int(x) for x in sub_end[:S]]
        keys = [out[ends[i]:ends[i + 1]].copy() for i in range(S)]
        return dict(keys=keys, subrounds=S, status=st)

    def decode_signed(self, max_rounds: int = 1 << 20):
        """Signed recovery of a set difference (count = +1 or -1 cells are pure);
        mutates the table.  Returns dict(keys=[array per round], signs=[int8 array
        per round], rounds=T, status=code); each round sorted by (key, sign)."""
        cap = int(max(1, np.abs(self.count).sum() + 1))
        cap = max(cap, self.n)
        out = np.zeros(cap, dtype=np.uint64)
        sg = np.zeros(cap, dtype=np.int8)
        mr = min(max_rounds, self.n + 2)
        round_end = np.zeros(mr + 1, dtype=np.uint64)
        T = np.zeros(1, dtype=np.uint32)
        st = lib().orc_iblt_decode_signed(self.n, self.r, self.seed, _ptr(self.count), _ptr(self.keyx),
                                          _ptr(self.chkx), mr, _ptr(out), _ptr(sg), cap, _ptr(round_end),
                                          _ptr(T))
        T = int(T[0])
        ends = [0] + [int(x) for x in round_end[:T]]
        return dict(keys=[out[ends[i]:ends[i + 1]].copy() for i in range(T)],
                    signs=[sg[ends[i]:ends[i + 1]].copy() for i in range(T)], rounds=T, status=st)

    def residual_cells(self) -> int:
        return int(np.count_nonzero(self.count))


# ----------------------------------------------------------------------------
# k-core on explicit hyperedges
# ----------------------------------------------------------------------------
def kcore_rounds(n: int, k: int, edges: np.ndarray, max_rounds: int = 1 << 30):
    """Round-synchronous peel.  Returns dict(vround, eround, s, m, rounds, status)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    m, r = (edges.shape if edges.ndim == 2 else (0, 1))
    vround = np.zeros(max(n, 1), dtype=np.int32)
    eround = np.zeros(max(m, 1), dtype=np.int32)
    mr = int(min(max_rounds, n + 1))
    s = np.zeros(mr + 1, dtype=np.uint64)
    mt = np.zeros(mr + 1, dtype=np.uint64)
    T = np.zeros(1, dtype=np.uint32)
    st = lib().orc_kcore_rounds(n, r, k, _ptr(edges), m, mr, _ptr(vround), _ptr(eround),
                                _ptr(s), _ptr(mt), _ptr(T))
    if st == INVALID:
        raise ValueError("invalid hypergraph (vertex id >= n)")
    T = int(T[0])
    return dict(vround=vround[:n], eround=eround[:m], s=[int(x) for x in s[:T]],
                m=[int(x) for x in mt[:T]], rounds=T, status=st)


def kcore_queue(n: int, k: int, edges: np.ndarray):
    """Sequential peel.  Returns (v_core uint8[n], e_core uint8[m])."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    m, r = (edges.shape if edges.ndim == 2 else (0, 1))
    vc = np.zeros(max(n, 1), dtype=np.uint8)
    ec = np.zeros(max(m, 1), dtype=np.uint8)
    st = lib().orc_kcore_queue(n, r, k, _ptr(edges), m, _ptr(vc), _ptr(ec))
    if st == INVALID:
        raise ValueError("invalid hypergraph (vertex id >= n)")
    return vc[:n], ec[:m]


def kcore_subrounds(n: int, k: int, edges: np.ndarray, part_off, max_subrounds: int = 1 << 30):
    """Peeling with sub-tables (App. B): part j = vertex ids part_off[j] ..
    part_off[j+1]-1, one part per sub-round.  Returns dict(vround, eround, s, m,
    subrounds, status) with s/m the vertices/edges left after each sub-round."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    m, r = (edges.shape if edges.ndim == 2 else (0, 1))
    off = np.ascontiguousarray(np.asarray(part_off, dtype=np.uint32))
    p = off.size - 1
    vround = np.zeros(max(n, 1), dtype=np.int32)
    eround = np.zeros(max(m, 1), dtype=np.int32)
    ms = int(min(max_subrounds, p * (n + 1)))
    s = np.zeros(ms + 1, dtype=np.uint64)
    mt = np.zeros(ms + 1, dtype=np.uint64)
    S = np.zeros(1, dtype=np.uint32)
    st = lib().orc_kcore_subrounds(n, r, k, _ptr(edges), m, p, _ptr(off), ms, _ptr(vround),
                                   _ptr(eround), _ptr(s), _ptr(mt), _ptr(S))
    if st == INVALID:
        raise ValueError("invalid hypergraph or parts")
    S = int(S[0])
    return dict(vround=vround[:n], eround=eround[:m], s=[int(x) for x in s[:S]],
                m=[int(x) for x in mt[:S]], subrounds=S, status=st)
