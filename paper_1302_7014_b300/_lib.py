"""ctypes declarations of libppeel.so (include/ppeel.h).

Loading fails loudly when the library has not been built: there is no other
implementation behind these names.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libppeel.so")

PP_MAX_R = 8

STATUS = {0: "PP_OK", 1: "PP_ERR_INVALID_ARG", 2: "PP_ERR_OUT_OF_MEMORY", 3: "PP_ERR_CAPACITY",
          4: "PP_ERR_ROUND_LIMIT", 5: "PP_ERR_TIMEOUT", 6: "PP_ERR_CUDA", 7: "PP_ERR_BUSY",
          8: "PP_ERR_NOT_FOUND"}

u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p


class Options(ctypes.Structure):
    _fields_ = [("block", u32), ("ctas_per_sm", u32), ("max_rounds", u32), ("host_loop", u32),
                ("stats_rounds", u32), ("binned", u32), ("kcore_mode", u32), ("rounds", u32), ("apply_ctas", u32),
                ("frontier_switch", u32), ("insert_chunk", u32), ("l2_fetch", u32)]


class DecodeResult(ctypes.Structure):
    _fields_ = [("rounds", u32), ("status_flags", u32), ("recovered", u64), ("items_before", u64),
                ("residual_cells", u64), ("round_cap", u32), ("pad", u32),
                ("recovered_per_round", ctypes.POINTER(u64)),
                ("remaining_per_round", ctypes.POINTER(u64)),
                ("alive_cells_per_round", ctypes.POINTER(u64))]


class PeelResult(ctypes.Structure):
    _fields_ = [("rounds", u32), ("status_flags", u32), ("core_vertices", u64), ("core_edges", u64),
                ("round_cap", u32), ("pad", u32), ("vertices_left", ctypes.POINTER(u64)),
                ("edges_left", ctypes.POINTER(u64))]


class Cell(ctypes.Structure):
    # see pp_cell: the key XOR, the checksum XOR and the count, one 32-byte sector
    _fields_ = [("key_xor", u64), ("chk_xor", u64), ("count", ctypes.c_int32), ("pad0", u32), ("pad1", u64)]


_SIGNATURES = {
    "pp_options_default": (None, [ctypes.POINTER(Options)]),
    "pp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pp_last_error": (ctypes.c_char_p, []),
    "pp_iblt_create": (ctypes.c_int, [ctypes.POINTER(vp), u64, u32, u64, ctypes.POINTER(Options)]),
    "pp_iblt_destroy": (ctypes.c_int, [vp]),
    "pp_iblt_clear": (ctypes.c_int, [vp, vp]),
    "pp_iblt_insert": (ctypes.c_int, [vp, vp, u64, vp]),
    "pp_iblt_delete": (ctypes.c_int, [vp, vp, u64, vp]),
    "pp_iblt_build": (ctypes.c_int, [vp, vp, u64, vp]),
    "pp_iblt_decode": (ctypes.c_int, [vp, vp, u64, ctypes.POINTER(DecodeResult), vp]),
    "pp_iblt_build_decode": (ctypes.c_int, [vp, vp, u64, vp, u64, ctypes.POINTER(DecodeResult), vp]),
    "pp_iblt_copy_cells": (ctypes.c_int, [vp, vp, u64, u64, ctypes.c_int, vp]),
    "pp_iblt_info": (ctypes.c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(u64)]),
    "pp_peel_kcore": (ctypes.c_int, [u32, u32, u32, vp, u64, vp, vp, ctypes.POINTER(PeelResult),
                                     ctypes.POINTER(Options), vp]),
    "pp_iblt_decode_subrounds": (ctypes.c_int, [vp, vp, u64, ctypes.POINTER(DecodeResult), vp]),
    "pp_workspace_size": (ctypes.c_int, [u64, u32, u64, ctypes.POINTER(Options), ctypes.POINTER(u64),
                                         ctypes.POINTER(u64), ctypes.POINTER(u64)]),
    "pp_iblt_decode_signed": (ctypes.c_int, [vp, vp, vp, u64, ctypes.POINTER(DecodeResult), vp]),
    "pp_peel_kcore_subrounds": (ctypes.c_int, [u32, u32, u32, vp, u64, u32, ctypes.POINTER(u32), vp, vp,
                                               ctypes.POINTER(PeelResult), ctypes.POINTER(Options), vp]),
    "pp_iblt_decode_noalloc": (ctypes.c_int, [vp, u64, u32, u64, vp, u64,
                                              ctypes.POINTER(DecodeResult), vp]),
    "pp_probe_scatter": (ctypes.c_int, [vp, u64, vp, u64, ctypes.c_int, vp]),
    "pp_iblt_submit_host": (ctypes.c_int, [vp, vp, u64, vp, u64, ctypes.POINTER(u64), vp]),
    "pp_iblt_finish_host": (ctypes.c_int, [vp, u64, ctypes.POINTER(DecodeResult)]),
    "pp_iblt_build_decode_host": (ctypes.c_int, [vp, vp, u64, vp, u64, ctypes.POINTER(DecodeResult), vp]),
}

PP_NOALLOC_MAX_CELLS = 1 << 20
PP_NOALLOC_MAX_ROUNDS = 4096

_lib = None


def load():
    """The loaded libppeel.so; raises if it was never built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_1302_7014_b300.build` "
                "(nvcc, sm_103a).  There is no fallback implementation.")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def declare(name: str, restype, argtypes):
    """Declare an additional entry point (used by the batch and server modules)."""
    _SIGNATURES[name] = (restype, argtypes)
    if _lib is not None:
        fn = getattr(_lib, name)
        fn.restype = restype
        fn.argtypes = argtypes
