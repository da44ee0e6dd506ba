"""Continuous-batching decode service (pp_server_* in include/ppeel.h)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, _lib
from ._lib import Options

u32, u64, i32, vp, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena_cells", u64), ("arena_keys", u64), ("max_slots", u32), ("max_queue", u32),
                ("r", u32), ("device", i32)]


class Request(ctypes.Structure):
    _fields_ = [("n_cells", u64), ("r", u32), ("pad", u32), ("table_seed", u64), ("m", u64),
                ("key_seed", u64), ("h_keys", vp), ("h_out", vp), ("out_cap", u64), ("arrival_s", dbl)]


class RequestResult(ctypes.Structure):
    _fields_ = [("ticket", u64), ("status", i32), ("rounds", u32), ("recovered", u64), ("items_before", u64),
                ("residual_cells", u64), ("arrival_s", dbl), ("admit_s", dbl), ("done_s", dbl)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, u64) for n in ("submitted", "admitted", "completed", "rejected", "pending", "active",
                                   "iterations", "keys_recovered", "iteration_us", "gpu_wait_us")]


_lib.declare("pp_server_now", dbl, [])
_lib.declare("pp_server_config_default", None, [ctypes.POINTER(ServerConfig)])
_lib.declare("pp_server_start", ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(ServerConfig),
                                               ctypes.POINTER(Options)])
_lib.declare("pp_server_submit", ctypes.c_int, [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)])
_lib.declare("pp_server_poll", ctypes.c_int, [vp, u64, ctypes.POINTER(RequestResult)])
_lib.declare("pp_server_wait", ctypes.c_int, [vp, u64, dbl, ctypes.POINTER(RequestResult)])
_lib.declare("pp_server_get_stats", ctypes.c_int, [vp, ctypes.POINTER(ServerStats)])
_lib.declare("pp_server_stop", ctypes.c_int, [vp, ctypes.c_int])

STATUS_BUSY = 7


def server_now() -> float:
    return _lib.load().pp_server_now()


class Server:
    """A running decode service.  Keep host key/output arrays alive until their request completes."""

    def __init__(self, arena_cells=1 << 26, arena_keys=1 << 26, max_slots=4096, r=0, device=0,
                 max_queue=0, opts: Options | None = None):
        lib = _lib.load()
        cfg = ServerConfig()
        lib.pp_server_config_default(ctypes.byref(cfg))
        cfg.arena_cells, cfg.arena_keys, cfg.max_slots, cfg.r, cfg.device = (
            int(arena_cells), int(arena_keys), int(max_slots), int(r), int(device))
        if max_queue:
            cfg.max_queue = int(max_queue)
        h = ctypes.c_void_p()
        _check(lib.pp_server_start(ctypes.byref(h), ctypes.byref(cfg),
                                   ctypes.byref(opts) if opts is not None else None), "pp_server_start")
        self._h = h
        self._keep = {}

    def submit(self, n_cells, r, table_seed, m, key_seed=0, keys: np.ndarray | None = None,
               want_keys=False, arrival_s=0.0) -> int:
        req = Request()
        req.n_cells, req.r, req.table_seed, req.m, req.key_seed = int(n_cells), int(r), int(table_seed) & (2**64 - 1), int(m), int(key_seed) & (2**64 - 1)
        req.arrival_s = float(arrival_s)
        keep = []
        if keys is not None:
            keys = np.ascontiguousarray(keys, dtype=np.uint64)
            req.h_keys = keys.ctypes.data
            keep.append(keys)
        out = None
        if want_keys:
            out = np.zeros(max(1, int(m)), dtype=np.uint64)
            req.h_out = out.ctypes.data
            req.out_cap = out.size
        t = u64()
        _check(_lib.load().pp_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "pp_server_submit")
        self._keep[t.value] = (keep, out)
        return t.value

    def _finish(self, ticket, res):
        keep, out = self._keep.pop(ticket, (None, None))
        d = {n: getattr(res, n) for n, _ in RequestResult._fields_}
        if out is not None:
            d["keys"] = out[: res.recovered].copy()
        return d

    def poll(self, ticket):
        res = RequestResult()
        st = _lib.load().pp_server_poll(self._h, ticket, ctypes.byref(res))
        if st == STATUS_BUSY:
            return None
        _check(st, "pp_server_poll")
        return self._finish(ticket, res)

    def wait(self, ticket, timeout_s=60.0):
        res = RequestResult()
        _check(_lib.load().pp_server_wait(self._h, ticket, float(timeout_s), ctypes.byref(res)), "pp_server_wait")
        return self._finish(ticket, res)

    def stats(self):
        s = ServerStats()
        _check(_lib.load().pp_server_get_stats(self._h, ctypes.byref(s)), "pp_server_get_stats")
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def stop(self, drain=True):
        if getattr(self, "_h", None) is not None and self._h.value:
            st = _lib.load().pp_server_stop(self._h, 1 if drain else 0)
            self._h = None
            _check(st, "pp_server_stop")

    def __del__(self):
        try:
            self.stop(drain=False)
        except Exception:
            pass


# Function-style names matching the C ABI.
def server_start(**kw) -> Server:
    return Server(**kw)
