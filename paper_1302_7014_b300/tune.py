"""Autotuner of the batched engine (pp_tune_batch) with an on-disk cache.

The search itself runs in the library (``csrc/tune.cu``): it times build +
decode of the caller's batch for each candidate setting of the run-time knobs
(ctas_per_sm, apply_ctas, binned, insert_chunk, rounds) and keeps the fastest one
whose per-table results equal the untuned run's.  This module remembers the
winner in a JSON file keyed by the GPU's name, the batch's ranks and size
buckets (log2 of its total cells and of its table count), so that later
batches of the same shape start from the tuned options without searching.

The cache lives at $PPEEL_TUNE_CACHE, else ~/.cache/ppeel/tune.json.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import tempfile
from dataclasses import dataclass, field

import numpy as np

from . import _check, _dev_ptr, _lib, _stream_ptr
from ._lib import Options
from .batch import Batch

u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p

TUNED_FIELDS = ("ctas_per_sm", "apply_ctas", "binned", "insert_chunk", "rounds")
MAX_CANDIDATES = 32


class TuneReport(ctypes.Structure):
    _fields_ = [("n_candidates", u32), ("best_index", u32), ("default_ms", ctypes.c_float),
                ("best_ms", ctypes.c_float), ("mismatches", u32), ("pad", u32)]


_lib.declare("pp_tune_batch", ctypes.c_int,
             [vp, vp, ctypes.POINTER(u64), vp, ctypes.POINTER(u64), u32, ctypes.POINTER(Options),
              ctypes.POINTER(TuneReport), ctypes.POINTER(ctypes.c_float), vp])


@dataclass
class TuneResult:
    options: dict                   # the tuned knobs
    default_ms: float | None        # untuned build + decode (None when taken from the cache)
    best_ms: float | None
    candidates_ms: list = field(default_factory=list)   # -1 = discarded (results differed)
    mismatches: int = 0
    from_cache: bool = False
    key: str = ""


def cache_path() -> str:
    return os.environ.get("PPEEL_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ppeel",
                                                            "tune.json"))


def shape_key(gpu_name: str, ranks, total_cells: int, n_tables: int) -> str:
    """Cache key: GPU name, the set of ranks, log2 buckets of cells and tables."""
    rs = "/".join(str(r) for r in sorted(set(int(x) for x in ranks)))
    cb = int(round(math.log2(max(1, int(total_cells)))))
    tb = int(round(math.log2(max(1, int(n_tables)))))
    return f"{gpu_name}|r={rs}|cells=2^{cb}|tables=2^{tb}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, options: dict, path: str | None = None, **info) -> None:
    """Writes one entry into the cache (atomic replace of the file)."""
    path = path or cache_path()
    data = load_cache(path)
    data[key] = dict(options=options, **info)
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".json", dir=d or ".")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def options_from(base: Options, tuned: dict) -> Options:
    o = Options()
    ctypes.memmove(ctypes.byref(o), ctypes.byref(base), ctypes.sizeof(Options))
    for k in TUNED_FIELDS:
        if k in tuned:
            setattr(o, k, int(tuned[k]))
    return o


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def tune_batch(batch: Batch, keys, key_offsets, out, out_offsets, reps: int = 3, use_cache: bool = True,
               path: str | None = None, stream=None) -> TuneResult:
    """Tuned options for ``batch`` (applied to it on return).  With use_cache,
    a cached entry for the batch's shape is applied without searching; a new
    search result is stored."""
    key = shape_key(_gpu_name(), batch.r, batch.total_cells(), batch.n_tables)
    if use_cache:
        hit = load_cache(path).get(key)
        if hit and all(k in hit.get("options", {}) for k in TUNED_FIELDS):
            batch.set_options(options_from(batch.options(), hit["options"]))
            return TuneResult(options=dict(hit["options"]), default_ms=None, best_ms=None, from_cache=True,
                              key=key)
    ko = np.ascontiguousarray(np.asarray(key_offsets, dtype=np.uint64))
    oo = np.ascontiguousarray(np.asarray(out_offsets, dtype=np.uint64))
    best = Options()
    rep = TuneReport()
    ms = (ctypes.c_float * MAX_CANDIDATES)()
    _check(_lib.load().pp_tune_batch(batch.handle, _dev_ptr(keys, 8, "keys"), ko.ctypes.data_as(ctypes.POINTER(u64)),
                                     _dev_ptr(out, 8, "out"), oo.ctypes.data_as(ctypes.POINTER(u64)), int(reps),
                                     ctypes.byref(best), ctypes.byref(rep), ms, _stream_ptr(stream)),
           "pp_tune_batch")
    opts = {k: int(getattr(best, k)) for k in TUNED_FIELDS}
    res = TuneResult(options=opts, default_ms=float(rep.default_ms), best_ms=float(rep.best_ms),
                     candidates_ms=[float(ms[i]) for i in range(rep.n_candidates)],
                     mismatches=int(rep.mismatches), key=key)
    if use_cache:
        store(key, opts, path, default_ms=res.default_ms, best_ms=res.best_ms)
    return res
