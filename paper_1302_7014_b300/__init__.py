"""Round-synchronous parallel peeling on one B300 (Python binding of libppeel.so).

Every operation runs in the CUDA kernels of ``libppeel.so``; this module only
marshals arguments (torch CUDA tensors for device memory, the current torch
stream) and turns status codes into exceptions.  Names follow the C ABI in
``include/ppeel.h``:

* ``IBLT`` / ``iblt_create``, ``iblt_insert``, ``iblt_delete``, ``iblt_decode``
  -- Invertible Bloom Lookup Tables (Sec. 6 of Jiang, Mitzenmacher & Thaler,
  "Parallel Peeling Algorithms"), decoded by round-synchronous peeling at k=2.
* ``peel_kcore`` -- round-synchronous k-core peeling of an explicit r-uniform
  hypergraph (Sec. 1, Sec. 3.1).
* ``IBLT.decode_subrounds`` / ``iblt_decode_subrounds`` and
  ``peel_kcore_subrounds`` -- the same processes with one part (sub-table) per
  sub-round, the order of the paper's GPU implementation (App. B).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

from . import _lib
from ._lib import PP_MAX_R, Cell, DecodeResult, Options, PeelResult

__all__ = ["PPError", "IBLT", "iblt_create", "iblt_insert", "iblt_delete", "iblt_build", "iblt_decode",
           "iblt_decode_subrounds", "iblt_decode_signed", "peel_kcore", "peel_kcore_subrounds", "options",
           "workspace_size", "PP_MAX_R", "CELL_DTYPE", "unpack_cells"]


class PPError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        self.status = status
        self.name = _lib.STATUS.get(status, f"status {status}")
        super().__init__(f"{fn}: {self.name}: {msg}")


# A pp_cell as stored on the device (32 bytes: key XOR, checksum XOR, count).
CELL_DTYPE = [("key_xor", "<u8"), ("chk_xor", "<u8"), ("count", "<i4"), ("pad0", "<u4"), ("pad1", "<u8")]


def unpack_cells(raw):
    """Stored cells (bytes or a CELL_DTYPE array) as a structured array with the
    fields key_xor, chk_xor and count."""
    import numpy as np
    if isinstance(raw, (bytes, bytearray, memoryview)):
        return np.frombuffer(raw, dtype=np.dtype(CELL_DTYPE))
    return np.asarray(raw).view(np.dtype(CELL_DTYPE))


def _check(status: int, fn: str):
    if status != 0:
        msg = _lib.load().pp_last_error()
        raise PPError(status, fn, msg.decode() if msg else "")


def workspace_size(n_cells: int, r: int, m_keys: int = 0, opts: Options | None = None) -> dict:
    """Device bytes of a table (pp_workspace_size): dict(table, fixed, peak)."""
    t, f, p = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.load().pp_workspace_size(int(n_cells), int(r), int(m_keys),
                                         ctypes.byref(opts) if opts is not None else None,
                                         ctypes.byref(t), ctypes.byref(f), ctypes.byref(p)), "pp_workspace_size")
    return {"table": t.value, "fixed": f.value, "peak": p.value}


def options(**kw) -> Options:
    """A pp_options struct with defaults, overridden by keyword arguments."""
    o = Options()
    _lib.load().pp_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(int(s.cuda_stream))


def _dev_ptr(t, elem_size: int, what: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.element_size() != elem_size:
        raise ValueError(f"{what} must have {elem_size}-byte elements")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class DecodeOutcome:
    rounds: int
    recovered: int
    items_before: int
    residual_cells: int
    status_flags: int
    recovered_per_round: list = field(default_factory=list)
    remaining_per_round: list = field(default_factory=list)
    alive_cells_per_round: list = field(default_factory=list)


@dataclass
class PeelOutcome:
    rounds: int
    core_vertices: int
    core_edges: int
    status_flags: int
    vertices_left: list = field(default_factory=list)
    edges_left: list = field(default_factory=list)


class IBLT:
    """An IBLT of ``n_cells`` cells and ``r`` hash functions on the current CUDA device."""

    def __init__(self, n_cells: int, r: int, seed: int, opts: Options | None = None):
        lib = _lib.load()
        h = ctypes.c_void_p()
        _check(lib.pp_iblt_create(ctypes.byref(h), int(n_cells), int(r), int(seed) & (2**64 - 1),
                                  ctypes.byref(opts) if opts is not None else None),
               "pp_iblt_create")
        self._h = h
        self.n_cells, self.r, self.seed = int(n_cells), int(r), int(seed)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().pp_iblt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def clear(self, stream=None):
        _check(_lib.load().pp_iblt_clear(self._h, _stream_ptr(stream)), "pp_iblt_clear")

    def insert(self, keys, stream=None):
        _check(_lib.load().pp_iblt_insert(self._h, _dev_ptr(keys, 8, "keys"), keys.numel(),
                                          _stream_ptr(stream)), "pp_iblt_insert")

    def delete(self, keys, stream=None):
        _check(_lib.load().pp_iblt_delete(self._h, _dev_ptr(keys, 8, "keys"), keys.numel(),
                                          _stream_ptr(stream)), "pp_iblt_delete")

    def build(self, keys, stream=None):
        """Clear the table and insert ``keys`` (one call, built slab by slab when large)."""
        _check(_lib.load().pp_iblt_build(self._h, _dev_ptr(keys, 8, "keys"), keys.numel(),
                                         _stream_ptr(stream)), "pp_iblt_build")

    def decode(self, out, round_cap: int = 4096, stream=None) -> DecodeOutcome:
        """Decode in place; ``out`` (CUDA, 8-byte elements) receives the keys."""
        return self._decode(_lib.load().pp_iblt_decode, "pp_iblt_decode", out, round_cap, stream)

    def build_decode(self, keys, out, round_cap: int = 4096, stream=None) -> DecodeOutcome:
        """build(keys) then decode(out) in one call; a large table's build
        then also finds the cells pure before round 1, and the decode does not
        scan the table again."""
        kp, n = _dev_ptr(keys, 8, "keys"), keys.numel()
        return self._decode(lambda h, o, cap, res, st: _lib.load().pp_iblt_build_decode(h, kp, n, o, cap, res, st),
                            "pp_iblt_build_decode", out, round_cap, stream)

    def decode_subrounds(self, out, round_cap: int = 4096, stream=None) -> DecodeOutcome:
        """Decode in place with one sub-table per sub-round (App. B); the per-round
        lists of the outcome are per sub-round."""
        return self._decode(_lib.load().pp_iblt_decode_subrounds, "pp_iblt_decode_subrounds", out,
                            round_cap, stream)

    def decode_signed(self, out, signs=None, round_cap: int = 4096, stream=None) -> DecodeOutcome:
        """Signed recovery of a set difference: ``out`` receives the keys and
        ``signs`` (CUDA int8, or None) +1 / -1 for each (Sec. 6 sparse recovery)."""
        sp = _dev_ptr(signs, 1, "signs")
        return self._decode(lambda h, o, cap, res, st: _lib.load().pp_iblt_decode_signed(h, o, sp, cap, res, st),
                            "pp_iblt_decode_signed", out, round_cap, stream)

    def submit_host(self, keys, out, stream=None) -> int:
        """Build from the host array ``keys`` (uint64) and decode, the recovered
        keys landing in the host array ``out``; returns a ticket for
        finish_host.  Both arrays must stay alive until then (pinned memory,
        e.g. a torch tensor made with pin_memory=True, is copied directly)."""
        import numpy as np
        keys = np.asarray(keys)
        out = np.asarray(out)
        if keys.dtype.itemsize != 8 or out.dtype.itemsize != 8 or not keys.flags.c_contiguous \
                or not out.flags.c_contiguous:
            raise ValueError("keys and out must be contiguous arrays of 8-byte elements")
        t = ctypes.c_uint64()
        _check(_lib.load().pp_iblt_submit_host(self._h, ctypes.c_void_p(keys.ctypes.data), keys.size,
                                               ctypes.c_void_p(out.ctypes.data), out.size, ctypes.byref(t),
                                               _stream_ptr(stream)), "pp_iblt_submit_host")
        self._host_jobs = getattr(self, "_host_jobs", {})
        self._host_jobs[t.value] = (keys, out)
        return t.value

    def finish_host(self, ticket: int, round_cap: int = 4096) -> DecodeOutcome:
        """Waits for a submit_host job; its outcome as decode() returns it."""
        try:
            return self._decode(lambda h, o, cap, res, st: _lib.load().pp_iblt_finish_host(h, ticket, res),
                                "pp_iblt_finish_host", None, round_cap, None)
        finally:
            getattr(self, "_host_jobs", {}).pop(ticket, None)

    def build_decode_host(self, keys, out, round_cap: int = 4096, stream=None) -> DecodeOutcome:
        return self.finish_host(self.submit_host(keys, out, stream), round_cap)

    def _decode(self, fn, name, out, round_cap, stream) -> DecodeOutcome:
        import numpy as np
        stats = np.empty((3, round_cap), dtype=np.uint64)  # filled up to the round count
        base = stats.ctypes.data
        res = DecodeResult()
        res.round_cap = round_cap
        res.recovered_per_round = ctypes.cast(base, ctypes.POINTER(ctypes.c_uint64))
        res.remaining_per_round = ctypes.cast(base + round_cap * 8, ctypes.POINTER(ctypes.c_uint64))
        res.alive_cells_per_round = ctypes.cast(base + 2 * round_cap * 8, ctypes.POINTER(ctypes.c_uint64))
        st = fn(self._h, _dev_ptr(out, 8, "out"), out.numel() if out is not None else 0, ctypes.byref(res),
                _stream_ptr(stream))
        _check(st, name)
        n = min(res.rounds, round_cap)
        return DecodeOutcome(res.rounds, res.recovered, res.items_before, res.residual_cells,
                             res.status_flags, stats[0, :n].tolist(), stats[1, :n].tolist(), stats[2, :n].tolist())

    def cells(self, stream=None):
        """Host copy of the table as a numpy structured array (key_xor, chk_xor,
        count); see unpack_cells."""
        import numpy as np
        out = np.zeros(self.n_cells, dtype=np.dtype(CELL_DTYPE))
        _check(_lib.load().pp_iblt_copy_cells(self._h, ctypes.c_void_p(out.ctypes.data), 0,
                                              self.n_cells, 1, _stream_ptr(stream)),
               "pp_iblt_copy_cells")
        return unpack_cells(out)

    def seeds(self) -> list[int]:
        n = ctypes.c_uint64()
        r = ctypes.c_uint32()
        s = (ctypes.c_uint64 * (PP_MAX_R + 1))()
        _check(_lib.load().pp_iblt_info(self._h, ctypes.byref(n), ctypes.byref(r), s), "pp_iblt_info")
        return list(s[: r.value + 1])


# Function-style names matching the C ABI.
def iblt_create(n_cells: int, r: int, seed: int, opts: Options | None = None) -> IBLT:
    return IBLT(n_cells, r, seed, opts)


def iblt_insert(table: IBLT, keys, stream=None) -> None:
    table.insert(keys, stream)


def iblt_delete(table: IBLT, keys, stream=None) -> None:
    table.delete(keys, stream)


def iblt_build(table: IBLT, keys, stream=None) -> None:
    table.build(keys, stream)


def iblt_decode(table: IBLT, out, round_cap: int = 4096, stream=None) -> DecodeOutcome:
    return table.decode(out, round_cap, stream)


def iblt_decode_subrounds(table: IBLT, out, round_cap: int = 4096, stream=None) -> DecodeOutcome:
    return table.decode_subrounds(out, round_cap, stream)


def iblt_decode_signed(table: IBLT, out, signs=None, round_cap: int = 4096, stream=None) -> DecodeOutcome:
    return table.decode_signed(out, signs, round_cap, stream)


def peel_kcore(n: int, r: int, k: int, edges, vertex_round=None, edge_round=None,
               opts: Options | None = None, round_cap: int = 4096, stream=None) -> PeelOutcome:
    """Peel the hypergraph ``edges`` ((m, r) CUDA tensor of 4-byte ids) to its k-core."""
    return _peel(n, r, k, edges, None, vertex_round, edge_round, opts, round_cap, stream)


def peel_kcore_subrounds(n: int, r: int, k: int, edges, part_off, vertex_round=None, edge_round=None,
                         opts: Options | None = None, round_cap: int = 4096,
                         stream=None) -> PeelOutcome:
    """Peel to the k-core with one part per sub-round (App. B): part j is vertex ids
    part_off[j] .. part_off[j+1]-1.  Rounds in the outcome are sub-rounds."""
    return _peel(n, r, k, edges, part_off, vertex_round, edge_round, opts, round_cap, stream)


def _peel(n, r, k, edges, part_off, vertex_round, edge_round, opts, round_cap, stream) -> PeelOutcome:
    m = edges.shape[0] if edges is not None and edges.numel() else 0
    if edges is not None and edges.numel() and (edges.dim() != 2 or edges.shape[1] != r):
        raise ValueError("edges must have shape (m, r)")
    import numpy as np
    stats = np.empty((2, round_cap), dtype=np.uint64)  # filled up to the round count
    res = PeelResult()
    res.round_cap = round_cap
    res.vertices_left = ctypes.cast(stats.ctypes.data, ctypes.POINTER(ctypes.c_uint64))
    res.edges_left = ctypes.cast(stats.ctypes.data + round_cap * 8, ctypes.POINTER(ctypes.c_uint64))
    common = (_dev_ptr(vertex_round, 4, "vertex_round"), _dev_ptr(edge_round, 4, "edge_round"),
              ctypes.byref(res), ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream))
    e_ptr = _dev_ptr(edges, 4, "edges") if m else None
    if part_off is None:
        st = _lib.load().pp_peel_kcore(int(n), int(r), int(k), e_ptr, int(m), *common)
        _check(st, "pp_peel_kcore")
    else:
        off = [int(x) for x in part_off]
        arr = (ctypes.c_uint32 * len(off))(*off)
        st = _lib.load().pp_peel_kcore_subrounds(int(n), int(r), int(k), e_ptr, int(m), len(off) - 1,
                                                 arr, *common)
        _check(st, "pp_peel_kcore_subrounds")
    nr = min(res.rounds, round_cap)
    return PeelOutcome(res.rounds, res.core_vertices, res.core_edges, res.status_flags,
                       stats[0, :nr].tolist(), stats[1, :nr].tolist())
