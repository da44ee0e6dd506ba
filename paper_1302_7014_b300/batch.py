"""Batched IBLT decode (pp_batch_* in include/ppeel.h): many tables, one graph launch."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from . import CELL_DTYPE, _check, _dev_ptr, _stream_ptr, unpack_cells
from ._lib import Options

u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p


class TableResult(ctypes.Structure):
    _fields_ = [("rounds", u32), ("stats_complete", u32), ("recovered", u64), ("items_before", u64),
                ("residual_cells", u64), ("round_cap", u32), ("pad", u32),
                ("recovered_per_round", ctypes.POINTER(u64))]


# The same record as a NumPy dtype: a batch's results are filled and read as
# columns instead of one ctypes object per table.
_RESULT_DTYPE = np.dtype([("rounds", "<u4"), ("stats_complete", "<u4"), ("recovered", "<u8"),
                          ("items_before", "<u8"), ("residual_cells", "<u8"), ("round_cap", "<u4"),
                          ("pad", "<u4"), ("recovered_per_round", "<u8")])
assert _RESULT_DTYPE.itemsize == ctypes.sizeof(TableResult)
assert all(_RESULT_DTYPE.fields[name][1] == getattr(TableResult, name).offset
           for name, _ in TableResult._fields_)


class PerRoundCounts:
    """recovered_per_round of a batch: entry i is table i's list of per-round
    counts, sliced from one (tables x round_cap) array when it is read."""

    def __init__(self, per_round: np.ndarray, rounds: np.ndarray):
        self._a = per_round
        self._n = np.minimum(rounds, per_round.shape[1])

    def __len__(self):
        return self._a.shape[0]

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        return self._a[i, : self._n[i]].tolist()

    def __iter__(self):
        return (self[i] for i in range(len(self)))


_lib.declare("pp_batch_create", ctypes.c_int, [ctypes.POINTER(vp), u32, ctypes.POINTER(u64),
                                               ctypes.POINTER(u32), ctypes.POINTER(u64),
                                               ctypes.POINTER(Options)])
_lib.declare("pp_batch_destroy", ctypes.c_int, [vp])
_lib.declare("pp_batch_clear", ctypes.c_int, [vp, vp])
_lib.declare("pp_batch_insert", ctypes.c_int, [vp, vp, ctypes.POINTER(u64), vp])
_lib.declare("pp_batch_delete", ctypes.c_int, [vp, vp, ctypes.POINTER(u64), vp])
_lib.declare("pp_batch_build", ctypes.c_int, [vp, vp, ctypes.POINTER(u64), vp])
_lib.declare("pp_batch_decode", ctypes.c_int, [vp, vp, ctypes.POINTER(u64), ctypes.POINTER(TableResult), vp])
_lib.declare("pp_batch_build_decode", ctypes.c_int,
             [vp, vp, ctypes.POINTER(u64), vp, ctypes.POINTER(u64), ctypes.POINTER(TableResult), vp])
_lib.declare("pp_batch_copy_cells", ctypes.c_int, [vp, u32, vp, ctypes.c_int, vp])
_lib.declare("pp_batch_info", ctypes.c_int, [vp, ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u32)])
_lib.declare("pp_batch_set_options", ctypes.c_int, [vp, ctypes.POINTER(Options)])
_lib.declare("pp_batch_get_options", ctypes.c_int, [vp, ctypes.POINTER(Options)])


@dataclass
class BatchOutcome:
    rounds: np.ndarray          # per table
    recovered: np.ndarray
    items_before: np.ndarray
    residual_cells: np.ndarray
    recovered_per_round: PerRoundCounts   # per table: list of per-round counts
    stats_complete: np.ndarray


def _u64_array(values):
    a = np.ascontiguousarray(np.asarray(values, dtype=np.uint64))
    return a, a.ctypes.data_as(ctypes.POINTER(u64))


class Batch:
    """n tables (sizes n_cells[i], ranks r[i], seeds seeds[i]) in one device arena."""

    def __init__(self, n_cells, r, seeds, opts: Options | None = None):
        lib = _lib.load()
        self.n_cells = [int(x) for x in n_cells]
        self.r = [int(x) for x in r]
        self.seeds = [int(x) & (2**64 - 1) for x in seeds]
        n = len(self.n_cells)
        nc, nc_p = _u64_array(self.n_cells)
        rr = np.ascontiguousarray(np.asarray(self.r, dtype=np.uint32))
        sd, sd_p = _u64_array(self.seeds)
        h = ctypes.c_void_p()
        _check(lib.pp_batch_create(ctypes.byref(h), n, nc_p, rr.ctypes.data_as(ctypes.POINTER(u32)), sd_p,
                                   ctypes.byref(opts) if opts is not None else None), "pp_batch_create")
        self._h = h
        self.n_tables = n
        self.stats_rounds = opts.stats_rounds if opts is not None and opts.stats_rounds else 128

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().pp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self, stream=None):
        _check(_lib.load().pp_batch_clear(self._h, _stream_ptr(stream)), "pp_batch_clear")

    def insert(self, keys, key_offsets, stream=None, sign: int = 1):
        """keys: CUDA tensor (8-byte elements); table i gets keys[key_offsets[i]:key_offsets[i+1]]."""
        off, off_p = _u64_array(key_offsets)
        assert off.size == self.n_tables + 1
        fn = _lib.load().pp_batch_insert if sign > 0 else _lib.load().pp_batch_delete
        ptr = _dev_ptr(keys, 8, "keys") if keys is not None and keys.numel() else None
        _check(fn(self._h, ptr, off_p, _stream_ptr(stream)), "pp_batch_insert")

    def delete(self, keys, key_offsets, stream=None):
        self.insert(keys, key_offsets, stream, sign=-1)

    def build(self, keys, key_offsets, stream=None):
        """Clear every table and insert ``keys`` (one call, slab by slab when large)."""
        off, off_p = _u64_array(key_offsets)
        assert off.size == self.n_tables + 1
        ptr = _dev_ptr(keys, 8, "keys") if keys is not None and keys.numel() else None
        _check(_lib.load().pp_batch_build(self._h, ptr, off_p, _stream_ptr(stream)), "pp_batch_build")

    def decode(self, out, out_offsets, round_cap: int = 256, stream=None) -> BatchOutcome:
        return self._decode(lambda ptr, off_p, res: _lib.load().pp_batch_decode(
            self._h, ptr, off_p, res, _stream_ptr(stream)), "pp_batch_decode", out, out_offsets, round_cap)

    def build_decode(self, keys, key_offsets, out, out_offsets, round_cap: int = 256,
                     stream=None) -> BatchOutcome:
        """build() then decode() in one call; a large batch's build then also
        finds the cells pure before round 1, and the decode does not scan the
        arena again."""
        koff, koff_p = _u64_array(key_offsets)
        assert koff.size == self.n_tables + 1
        kptr = _dev_ptr(keys, 8, "keys") if keys is not None and keys.numel() else None
        return self._decode(lambda ptr, off_p, res: _lib.load().pp_batch_build_decode(
            self._h, kptr, koff_p, ptr, off_p, res, _stream_ptr(stream)), "pp_batch_build_decode", out,
            out_offsets, round_cap)

    def _decode(self, call, name, out, out_offsets, round_cap) -> BatchOutcome:
        off, off_p = _u64_array(out_offsets)
        n = self.n_tables
        per_round = np.zeros((n, round_cap), dtype=np.uint64)
        results = np.zeros(n, dtype=_RESULT_DTYPE)
        results["round_cap"] = round_cap
        results["recovered_per_round"] = (np.uint64(per_round.ctypes.data)
                                          + np.arange(n, dtype=np.uint64) * np.uint64(round_cap * 8))
        ptr = _dev_ptr(out, 8, "out") if out is not None and out.numel() else None
        _check(call(ptr, off_p, ctypes.cast(results.ctypes.data, ctypes.POINTER(TableResult))), name)
        rounds = results["rounds"].astype(np.int64)
        return BatchOutcome(
            rounds=rounds,
            recovered=results["recovered"].astype(np.int64),
            items_before=results["items_before"].astype(np.int64),
            residual_cells=results["residual_cells"].astype(np.int64),
            recovered_per_round=PerRoundCounts(per_round, rounds),
            stats_complete=results["stats_complete"].astype(bool))

    def set_options(self, opts: Options) -> None:
        _check(_lib.load().pp_batch_set_options(self._h, ctypes.byref(opts)), "pp_batch_set_options")

    def options(self) -> Options:
        o = Options()
        _check(_lib.load().pp_batch_get_options(self._h, ctypes.byref(o)), "pp_batch_get_options")
        return o

    @property
    def handle(self):
        return self._h

    def total_cells(self) -> int:
        n = u32()
        c = u64()
        _check(_lib.load().pp_batch_info(self._h, ctypes.byref(n), ctypes.byref(c), None), "pp_batch_info")
        return int(c.value)

    def cells(self, table: int):
        out = np.zeros(self.n_cells[table], dtype=np.dtype(CELL_DTYPE))
        _check(_lib.load().pp_batch_copy_cells(self._h, table, ctypes.c_void_p(out.ctypes.data), 1,
                                               _stream_ptr(None)), "pp_batch_copy_cells")
        return unpack_cells(out)


# Function-style names matching the C ABI.
def batch_create(n_cells, r, seeds, opts: Options | None = None) -> Batch:
    return Batch(n_cells, r, seeds, opts)


def batch_insert(batch: Batch, keys, key_offsets, stream=None) -> None:
    batch.insert(keys, key_offsets, stream)


def batch_build(batch: Batch, keys, key_offsets, stream=None) -> None:
    batch.build(keys, key_offsets, stream)


def batch_decode(batch: Batch, out, out_offsets, round_cap: int = 256, stream=None) -> BatchOutcome:
    return batch.decode(out, out_offsets, round_cap, stream)
