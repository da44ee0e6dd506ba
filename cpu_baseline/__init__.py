"""CPU baseline: the round-synchronous IBLT build and decode on every host core
(OpenMP, ``rounds_omp.c``).  Used by ``bench.py``'s CPU baseline and checked
against the oracle in the tests; the library never touches it."""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rounds_omp.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librounds_omp.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
        os.close(fd)
        subprocess.check_call(["gcc", "-O3", "-march=native", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        so = ctypes.CDLL(build())
        u64, u32, vp, i = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
        so.omp_threads.restype = i
        so.omp_iblt_build.argtypes = [u64, u32, u64, vp, u64, vp, vp, vp, i]
        so.omp_iblt_build.restype = i
        so.omp_iblt_decode.argtypes = [u64, u32, u64, vp, vp, vp, u32, vp, u64, vp, vp, i]
        so.omp_iblt_decode.restype = i
        _lib = so
    return _lib


def threads() -> int:
    return int(lib().omp_threads())


def build_and_decode(n: int, r: int, table_seed: int, keys: np.ndarray, n_threads: int = 0,
                     max_rounds: int = 1 << 20):
    """Returns dict(keys=[array per round], rounds, build_s, decode_s, count, keyx, chkx, status)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    cnt = np.zeros(n, np.int64)
    kx = np.zeros(n, np.uint64)
    cx = np.zeros(n, np.uint64)
    so = lib()
    t0 = time.perf_counter()
    st = so.omp_iblt_build(n, r, table_seed, keys.ctypes.data, keys.size, cnt.ctypes.data, kx.ctypes.data,
                           cx.ctypes.data, int(n_threads))
    t1 = time.perf_counter()
    if st:
        raise ValueError(f"omp_iblt_build status {st}")
    out = np.zeros(max(1, keys.size), np.uint64)
    mr = int(min(max_rounds, n + 2))
    ends = np.zeros(mr + 1, np.uint64)
    T = np.zeros(1, np.uint32)
    st = so.omp_iblt_decode(n, r, table_seed, cnt.ctypes.data, kx.ctypes.data, cx.ctypes.data, mr, out.ctypes.data,
                            out.size, ends.ctypes.data, T.ctypes.data, int(n_threads))
    t2 = time.perf_counter()
    T = int(T[0])
    e = [0] + [int(x) for x in ends[:T]]
    return dict(keys=[out[e[i]:e[i + 1]].copy() for i in range(T)], rounds=T, build_s=t1 - t0,
                decode_s=t2 - t1, count=cnt, keyx=kx, chkx=cx, status=st)
