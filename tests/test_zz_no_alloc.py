"""pp_iblt_decode_noalloc against pp_iblt_decode, through the C ABI.

The no-allocation decode is for callers that may not allocate device memory
while they run (a framework that has reserved the GPU's memory for its own
pool, a no-allocation-after-start-up rule, or code that cannot take cudaFree's
device-wide synchronisation).  It keeps its working memory in one fixed array
in the library's device code, shared by every call; these checks run two calls
in a row, so the second one starts from the first one's leftovers.

This file is collected last on purpose; it must pass both on its own in a
fresh process and after the other tests.
"""
import ctypes
import gc

import numpy as np
import pytest

import ppgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _result(round_cap):
    from paper_1302_7014_b300 import _lib
    arrays = [(ctypes.c_uint64 * round_cap)() for _ in range(3)]
    res = _lib.DecodeResult()
    res.round_cap = round_cap
    res.recovered_per_round = ctypes.cast(arrays[0], ctypes.POINTER(ctypes.c_uint64))
    res.remaining_per_round = ctypes.cast(arrays[1], ctypes.POINTER(ctypes.c_uint64))
    res.alive_cells_per_round = ctypes.cast(arrays[2], ctypes.POINTER(ctypes.c_uint64))
    return res, arrays


def _by_round(keys, counts):
    ends = np.cumsum([0] + list(counts))
    return [np.sort(keys[ends[i]:ends[i + 1]]) for i in range(len(counts))]


def _one_case(lib, pp, n, r, c, seed, key_seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), key_seed)
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    ref = pp.IBLT(n, r, seed)
    ref.insert(dkeys)
    # the caller's own copy of the built table, in caller-owned device memory
    cells = torch.empty(n * ctypes.sizeof(pp._lib.Cell), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.pp_iblt_copy_cells(ref.handle, ctypes.c_void_p(cells.data_ptr()), 0, n, 0, stream) == 0
    # existing entry point
    out_ref = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    want = ref.decode(out_ref)
    # no-allocation entry point, through the C ABI
    out = torch.full((keys.size,), -1, dtype=torch.int64, device="cuda")
    res, arrays = _result(4096)
    st = lib.pp_iblt_decode_noalloc(ctypes.c_void_p(cells.data_ptr()), n, r, seed,
                                    ctypes.c_void_p(out.data_ptr()), keys.size, ctypes.byref(res),
                                    stream)
    assert st == 0, lib.pp_last_error()
    T = res.rounds
    assert T == want.rounds
    assert res.recovered == want.recovered and res.items_before == want.items_before
    assert res.residual_cells == want.residual_cells
    assert list(arrays[0][:T]) == want.recovered_per_round
    assert list(arrays[1][:T]) == want.remaining_per_round
    assert list(arrays[2][:T]) == want.alive_cells_per_round
    got = out[: res.recovered].cpu().numpy().view(np.uint64)
    ref_keys = out_ref[: want.recovered].cpu().numpy().view(np.uint64)
    for a, b in zip(_by_round(got, want.recovered_per_round), _by_round(ref_keys, want.recovered_per_round)):
        assert (a == b).all()
    # the decoded-in-place tables are identical too
    after = pp.unpack_cells(cells.cpu().numpy().view(np.dtype(pp.CELL_DTYPE)))
    assert (after == ref.cells()).all()
    ref.close()


def test_noalloc_matches_decode_two_calls_in_a_row(ppeel_lib):
    import paper_1302_7014_b300 as pp
    lib = ppeel_lib
    # two calls in a row: the second reuses the first one's scratch contents
    _one_case(lib, pp, 300007, 3, 0.75, 17, 18)
    _one_case(lib, pp, 65539, 4, 0.85, 19, 20)   # above threshold: non-empty residue
    _one_case(lib, pp, 1 << 20, 3, 0.80, 21, 22)  # the largest table it accepts


def test_noalloc_calls_allocate_no_device_memory(ppeel_lib):
    # After the first call on the device (which loads the library's device
    # code, see the header), further calls leave the free device memory and
    # torch's own allocations exactly as they were.
    import paper_1302_7014_b300 as pp
    lib = ppeel_lib
    n, r, seed = 200003, 3, 29
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.75, n), 30)
    dkeys = torch.from_numpy(keys.view(np.int64)).cuda()
    ref = pp.IBLT(n, r, seed)
    ref.insert(dkeys)
    cells = torch.empty(n * ctypes.sizeof(pp._lib.Cell), dtype=torch.uint8, device="cuda")
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    res, _ = _result(1024)

    def call():
        assert lib.pp_iblt_copy_cells(ref.handle, ctypes.c_void_p(cells.data_ptr()), 0, n, 0, stream) == 0
        st = lib.pp_iblt_decode_noalloc(ctypes.c_void_p(cells.data_ptr()), n, r, seed,
                                        ctypes.c_void_p(out.data_ptr()), keys.size, ctypes.byref(res), stream)
        assert st == 0, lib.pp_last_error()
        assert res.recovered == keys.size
        torch.cuda.synchronize()

    call()   # warm-up: the first call may load the module
    # no Python garbage collection (which could free unrelated tensors) while measuring
    gc.collect()
    gc.disable()
    try:
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        for _ in range(3):
            call()
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
    finally:
        gc.enable()
    ref.close()


def test_noalloc_rejects_misaligned_cells(ppeel_lib):
    res, _ = _result(16)
    buf = torch.zeros(64 * 32 + 16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    st = ppeel_lib.pp_iblt_decode_noalloc(ctypes.c_void_p(buf.data_ptr() + 16), 64, 3, 1,
                                          ctypes.c_void_p(out.data_ptr()), 8, ctypes.byref(res), None)
    from paper_1302_7014_b300 import _lib
    assert _lib.STATUS[st] == "PP_ERR_INVALID_ARG"
    assert b"aligned" in ppeel_lib.pp_last_error()


def test_noalloc_rejects_oversized_table(ppeel_lib):
    from paper_1302_7014_b300 import _lib
    res, _ = _result(16)
    dummy = torch.zeros(32, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    st = ppeel_lib.pp_iblt_decode_noalloc(ctypes.c_void_p(dummy.data_ptr()), _lib.PP_NOALLOC_MAX_CELLS + 1,
                                          3, 1, ctypes.c_void_p(out.data_ptr()), 8, ctypes.byref(res),
                                          None)
    assert _lib.STATUS[st] == "PP_ERR_INVALID_ARG"
    assert b"PP_NOALLOC_MAX_CELLS" in ppeel_lib.pp_last_error()
