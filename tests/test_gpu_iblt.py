"""GPU parity: IBLT build and round-synchronous decode against the CPU oracle.

Every comparison is exact (integer/XOR work): the built table bit for bit,
each round's recovered key set, the number of rounds, the per-round survivor
counts and the residue left in the table.  Sizes span several scan chunks
(1024 cells) and peel chunks (512 entries) with ragged tails.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import ppgen
from conftest import GOLDEN

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pp(ppeel_lib):
    import paper_1302_7014_b300 as pp
    return pp


def _dev(keys):
    return torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()


def _split_rounds(out_keys, rec_per_round):
    ends = np.cumsum([0] + list(rec_per_round))
    return [np.sort(out_keys[ends[i]:ends[i + 1]]) for i in range(len(rec_per_round))]


def _assert_cells_equal(cells, ot):
    assert (cells["count"].astype(np.int64) == ot.count).all()
    assert (cells["key_xor"] == ot.keyx).all()
    assert (cells["chk_xor"] == ot.chkx).all()


def run_case(pp, n, r, keys, seed, opts=None, deletes=None, max_rounds=None):
    """Build and decode on the GPU and in the oracle; compare everything."""
    gt = pp.IBLT(n, r, seed, opts)
    ot = oracle.IBLT(n, r, seed)
    if len(keys):
        gt.insert(_dev(keys))
    ot.insert(keys)
    if deletes is not None and len(deletes):
        gt.delete(_dev(deletes))
        ot.insert(deletes, sign=-1)
    torch.cuda.synchronize()
    _assert_cells_equal(gt.cells(), ot)                     # build parity
    items = len(keys) - (0 if deletes is None else len(deletes))
    out = torch.zeros(max(1, items), dtype=torch.int64, device="cuda")
    res = gt.decode(out)
    ores = ot.decode_rounds() if max_rounds is None else ot.decode_rounds(max_rounds=max_rounds)
    assert res.rounds == ores["rounds"]
    got = out[: res.recovered].cpu().numpy().view(np.uint64)
    rounds = _split_rounds(got, res.recovered_per_round)
    assert len(rounds) == len(ores["keys"])
    for t, (a, b) in enumerate(zip(rounds, ores["keys"])):
        assert a.size == b.size, f"round {t + 1}"
        assert (a == np.sort(b)).all(), f"round {t + 1}"
    assert res.alive_cells_per_round == ores["cells_alive"]
    left = items - np.cumsum([k.size for k in ores["keys"]])
    assert res.remaining_per_round == [int(x) for x in left]
    _assert_cells_equal(gt.cells(), ot)                     # residue parity
    assert res.residual_cells == ot.residual_cells()
    gt.close()
    return res, ores


CASES = [
    # n_cells, r, load c, seed
    (1000, 3, 0.70, 1),
    (3 * 1024 + 17, 3, 0.75, 2),
    (65541, 3, 0.75, 3),
    (65536, 4, 0.70, 4),
    (50000, 4, 0.85, 5),        # above c*_{2,4}: non-empty core
    (20000, 3, 0.90, 6),        # above c*_{2,3}
    (7777, 2, 0.40, 7),         # r = 2 (generic kernels)
    (4099, 5, 0.60, 8),
    (3001, 8, 0.50, 9),
    (256, 3, 0.70, 10),
    (200003, 3, 1.20, 12),      # far above threshold
    ((1 << 20) + 13, 3, 0.80, 13),
    ((1 << 18) + 1, 4, 0.76, 14),
]


@pytest.mark.parametrize("n,r,c,seed", CASES, ids=[f"n{n}-r{r}-c{c}" for n, r, c, _ in CASES])
def test_iblt_parity(pp, n, r, c, seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 1000 + seed)
    run_case(pp, n, r, keys, seed)


@pytest.mark.parametrize("n,r,c,seed", CASES[:6], ids=[f"hostloop-n{n}-r{r}" for n, r, c, _ in CASES[:6]])
def test_iblt_parity_host_loop(pp, n, r, c, seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 2000 + seed)
    run_case(pp, n, r, keys, seed, opts=pp.options(host_loop=1))


def test_small_grid_many_chunks_per_cta(pp):
    # one CTA per SM forces every kernel through several grid-stride chunks
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.78, 300007), 77)
    run_case(pp, 300007, 3, keys, 21, opts=pp.options(ctas_per_sm=1))


def test_empty_table(pp):
    res, _ = run_case(pp, 100, 3, np.zeros(0, np.uint64), 5)
    assert res.rounds == 0 and res.recovered == 0 and res.residual_cells == 0


def test_minimum_table_and_single_key(pp):
    run_case(pp, 3, 3, ppgen.distinct_keys(1, 9), 9)
    run_case(pp, 30, 3, ppgen.distinct_keys(1, 10), 10)
    run_case(pp, 3, 3, ppgen.distinct_keys(2, 11), 11)


def test_duplicate_cells_leave_a_core(pp):
    n, r, seed = 9, 3, 77
    cand = ppgen.distinct_keys(200000, 5)
    cells = oracle.key_cells(n, r, seed, cand)
    seen, pair = {}, None
    for x, row in zip(cand.tolist(), map(tuple, cells.tolist())):
        if row in seen:
            pair = (seen[row], x)
            break
        seen[row] = x
    res, _ = run_case(pp, n, r, np.array(pair, np.uint64), seed)
    assert res.rounds == 0 and res.residual_cells == 3


def test_deletions(pp):
    keys = ppgen.distinct_keys(30000, 31)
    dele = keys[::3].copy()
    run_case(pp, 50000, 3, keys, 31, deletes=dele)


@pytest.mark.parametrize("n,binned", [(50000, 2), (1 << 22, 1)])
def test_deleting_keys_never_inserted(pp, n, binned):
    """Cells left with negative counts: the residue count is every cell with a
    non-zero count, as in the oracle (a count can go from 0 to -1 while keys
    are deleted from the table during the decode)."""
    r, seed = 3, 61
    keys = ppgen.distinct_keys(int(0.6 * n), 62)
    ghost = ppgen.distinct_keys(int(0.05 * n), 63)
    gt = pp.IBLT(n, r, seed, pp.options(binned=binned))
    ot = oracle.IBLT(n, r, seed)
    gt.insert(_dev(keys))
    gt.delete(_dev(ghost))
    ot.insert(keys)
    ot.insert(ghost, sign=-1)
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    res = gt.decode(out)
    ores = ot.decode_rounds()
    assert res.rounds == ores["rounds"]
    assert res.recovered_per_round == [k.size for k in ores["keys"]]
    _assert_cells_equal(gt.cells(), ot)
    assert res.residual_cells == ot.residual_cells()


@pytest.mark.parametrize("binned,host_loop,rounds", [(2, 0, 0), (1, 0, 1), (1, 1, 1), (0, 0, 2), (0, 1, 2)],
                         ids=["rounds", "binned", "binned-hostloop", "tiles", "tiles-hostloop"])
def test_round_limit(pp, binned, host_loop, rounds):
    """A decode stopped by the round limit leaves the table as the oracle's after that round.
    In the binned decode this also checks the end-of-decode clearing of the winners' cells:
    the frontier that was found but not processed must stay untouched."""
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.80, 100000), 41)
    opts = pp.options(max_rounds=3, binned=binned, host_loop=host_loop, rounds=rounds)
    with pytest.raises(pp.PPError) as ei:
        run_case(pp, 100000, 3, keys, 41, opts=opts, max_rounds=3)
    assert ei.value.name == "PP_ERR_ROUND_LIMIT"
    # the table is left after round 3, like the oracle's
    gt = pp.IBLT(100000, 3, 41, opts)
    ot = oracle.IBLT(100000, 3, 41)
    gt.insert(_dev(keys))
    ot.insert(keys)
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError):
        gt.decode(out)
    ores = ot.decode_rounds(max_rounds=3)
    assert ores["status"] == oracle.ROUND_LIMIT and ores["rounds"] == 3
    _assert_cells_equal(gt.cells(), ot)


def test_capacity_checked_before_decoding(pp):
    keys = ppgen.distinct_keys(1000, 51)
    gt = pp.IBLT(2000, 3, 51)
    gt.insert(_dev(keys))
    before = gt.cells().copy()
    out = torch.zeros(999, dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError) as ei:
        gt.decode(out)
    assert ei.value.name == "PP_ERR_CAPACITY"
    assert (gt.cells() == before).all()


def test_decode_twice_and_reuse(pp):
    n, r, seed = 40000, 3, 61
    gt = pp.IBLT(n, r, seed)
    for rep in range(3):
        keys = ppgen.distinct_keys(ppgen.edges_from_c(0.7, n), 6100 + rep)
        gt.clear()
        gt.insert(_dev(keys))
        out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
        res = gt.decode(out)
        got = np.sort(out[: res.recovered].cpu().numpy().view(np.uint64))
        ot = oracle.IBLT(n, r, seed)
        ot.insert(keys)
        ores = ot.decode_rounds()
        assert res.rounds == ores["rounds"]
        assert (got == np.sort(np.concatenate(ores["keys"]))).all()
        res2 = gt.decode(out)     # nothing left to recover
        assert res2.rounds == 0 and res2.recovered == 0


def test_invalid_arguments(pp):
    with pytest.raises(pp.PPError) as ei:
        pp.IBLT(100, 1, 0)
    assert ei.value.name == "PP_ERR_INVALID_ARG"
    with pytest.raises(pp.PPError):
        pp.IBLT(100, 9, 0)
    with pytest.raises(pp.PPError):
        pp.IBLT(2, 3, 0)


def test_seeds_match_convention(pp):
    gt = pp.IBLT(1000, 4, 0x1234)
    assert gt.seeds() == [int(s) for s in oracle.hash_seeds(0x1234, 4)]


@pytest.mark.parametrize("fused", [False, True], ids=["insert-decode", "build_decode"])
def test_headline_full_size(pp, fused):
    """2^26 cells, r = 3, load 0.75 against the oracle's stored trajectory:
    insert then decode, and the benchmark's one-call build + decode (whose
    build finds F_1)."""
    gold = json.load(open(os.path.join(GOLDEN, "full_size.json")))["iblt_headline"]
    n, r, m = gold["n_cells"], gold["r"], gold["m"]
    keys = ppgen.distinct_keys(m, gold["key_seed"])
    gt = pp.IBLT(n, r, gold["table_seed"])
    dkeys = _dev(keys)
    out = torch.zeros(m, dtype=torch.int64, device="cuda")
    if fused:
        res = gt.build_decode(dkeys, out)
    else:
        gt.insert(dkeys)
        res = gt.decode(out)
    assert res.rounds == gold["rounds"]
    assert res.recovered_per_round == gold["recovered_per_round"]
    assert res.alive_cells_per_round == gold["alive_cells_per_round"]
    assert res.residual_cells == gold["residual_cells"] == 0
    got = out.cpu().numpy().view(np.uint64)
    rounds = _split_rounds(got, res.recovered_per_round)
    for t, (a, h) in enumerate(zip(rounds, gold["round_sha256"])):
        assert hashlib.sha256(a.tobytes()).hexdigest() == h, f"round {t + 1}"
    assert (np.sort(got) == np.sort(keys)).all()   # recovered set == inserted set


@pytest.mark.parametrize("n,r,c", [(3 * (1 << 21) + 17, 3, 0.75), ((1 << 22) + 5, 4, 0.7), (5000, 3, 0.8),
                                   (70001, 5, 0.6)])
def test_binned_build_insert_delete(pp, n, r, c):
    """The slab-binned update paths (forced on) against the oracle, cell for cell."""
    seed = n + r
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), seed + 1)
    dk = _dev(keys)
    # build from scratch (zero-filled slab by slab)
    gt = pp.IBLT(n, r, seed, pp.options(binned=1))
    gt.insert(_dev(ppgen.distinct_keys(1000, 5)))   # junk that build() must wipe
    gt.build(dk)
    ot = oracle.IBLT(n, r, seed)
    ot.insert(keys)
    _assert_cells_equal(gt.cells(), ot)
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    res = gt.decode(out)
    ores = ot.decode_rounds()
    assert res.rounds == ores["rounds"] and res.recovered_per_round == [k.size for k in ores["keys"]]
    _assert_cells_equal(gt.cells(), ot)
    # incremental inserts and a delete on a non-empty table
    gt.clear()
    half = keys.size // 2
    gt.insert(_dev(keys[:half]))
    gt.insert(_dev(keys[half:]))
    gt.delete(_dev(keys[::5]))
    ot2 = oracle.IBLT(n, r, seed)
    ot2.insert(keys)
    ot2.insert(keys[::5], sign=-1)
    _assert_cells_equal(gt.cells(), ot2)
    gt.close()


def test_build_without_binning_matches(pp):
    n, r = 100000, 3
    keys = ppgen.distinct_keys(70000, 3)
    gt = pp.IBLT(n, r, 9, pp.options(binned=2))
    gt.build(_dev(keys))
    ot = oracle.IBLT(n, r, 9)
    ot.insert(keys)
    _assert_cells_equal(gt.cells(), ot)


def test_headline_full_size_build(pp):
    """The benchmark's step (build + decode) at 2^26 cells against the stored oracle trajectory."""
    gold = json.load(open(os.path.join(GOLDEN, "full_size.json")))["iblt_headline"]
    n, r, m = gold["n_cells"], gold["r"], gold["m"]
    keys = ppgen.distinct_keys(m, gold["key_seed"])
    gt = pp.IBLT(n, r, gold["table_seed"])
    dkeys = _dev(keys)
    out = torch.zeros(m, dtype=torch.int64, device="cuda")
    for _ in range(2):                                    # twice: workspace reuse
        gt.build(dkeys)
        res = gt.decode(out)
        assert res.rounds == gold["rounds"]
        assert res.recovered_per_round == gold["recovered_per_round"]
        assert res.alive_cells_per_round == gold["alive_cells_per_round"]
        assert res.residual_cells == 0
    got = out.cpu().numpy().view(np.uint64)
    rounds = _split_rounds(got, res.recovered_per_round)
    for t, (a, h) in enumerate(zip(rounds, gold["round_sha256"])):
        assert hashlib.sha256(a.tobytes()).hexdigest() == h, f"round {t + 1}"


BINNED_CASES = CASES + [(3 * (1 << 19) + 17, 3, 0.75, 31), ((1 << 21) + 1, 4, 0.85, 32),
                        (5 * (1 << 19) - 3, 5, 0.6, 33)]


@pytest.mark.parametrize("n,r,c,seed", BINNED_CASES, ids=[f"binned-n{n}-r{r}-c{c}" for n, r, c, _ in BINNED_CASES])
def test_iblt_parity_binned_rounds(pp, n, r, c, seed):
    """Rounds split into claim + address-ordered apply (forced on) against the oracle."""
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 3000 + seed)
    run_case(pp, n, r, keys, seed, opts=pp.options(binned=1, rounds=1))


@pytest.mark.parametrize("n,r,c,seed", BINNED_CASES[-3:], ids=[f"binned-hostloop-n{n}" for n, r, c, _ in BINNED_CASES[-3:]])
def test_iblt_parity_binned_rounds_host_loop(pp, n, r, c, seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 4000 + seed)
    run_case(pp, n, r, keys, seed, opts=pp.options(binned=1, host_loop=1, ctas_per_sm=1, rounds=1))


def test_binned_rounds_after_workspace_growth(pp):
    # a small build first, then a bigger one: the record buffers move and the
    # decode graph must follow them
    n, r = 3 * (1 << 19) + 5, 3
    gt = pp.IBLT(n, r, 5, pp.options(binned=1, rounds=1))
    for m_frac in (0.1, 0.8, 0.75):
        keys = ppgen.distinct_keys(ppgen.edges_from_c(m_frac, n), int(m_frac * 100))
        gt.build(_dev(keys))
        out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
        res = gt.decode(out)
        ot = oracle.IBLT(n, r, 5)
        ot.insert(keys)
        ores = ot.decode_rounds()
        assert res.rounds == ores["rounds"]
        assert res.recovered_per_round == [k.size for k in ores["keys"]]
        _assert_cells_equal(gt.cells(), ot)


def test_workspace_size_matches_allocations(pp):
    """pp_workspace_size against the device memory a handle really takes."""
    n, r = 1 << 24, 3
    m = int(0.75 * n)
    ws = pp.workspace_size(n, r, m)
    keys = _dev(ppgen.distinct_keys(m, 71))
    out = torch.zeros(m, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t = pp.IBLT(n, r, 72)
    free1 = torch.cuda.mem_get_info()[0]
    t.build(keys)
    res = t.decode(out)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert res.recovered == m
    slack = (64 << 20) + ws["peak"] // 50   # allocation granularity, graph and context memory
    assert abs((free0 - free1) - (ws["table"] + ws["fixed"])) < slack
    assert abs((free0 - free2) - ws["peak"]) < slack
    t.close()


# ---- tile rounds: each round's updates folded per 4096-cell tile ------------
TILE_CASES = CASES + [((1 << 21) + 1, 4, 0.85, 32), (3 * (1 << 21) + 17, 3, 0.75, 34)]


@pytest.mark.parametrize("n,r,c,seed", TILE_CASES, ids=[f"tiles-n{n}-r{r}-c{c}" for n, r, c, _ in TILE_CASES])
def test_iblt_parity_tile_rounds(pp, n, r, c, seed):
    """Tile rounds (forced on for any size) against the oracle: per-round key
    sets, survivors, the residue cell for cell."""
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 5000 + seed)
    run_case(pp, n, r, keys, seed, opts=pp.options(rounds=2))


@pytest.mark.parametrize("n,r,c,seed", TILE_CASES[:6] + TILE_CASES[-2:],
                         ids=[f"tiles-hostloop-n{n}-r{r}" for n, r, c, _ in TILE_CASES[:6] + TILE_CASES[-2:]])
def test_iblt_parity_tile_rounds_host_loop(pp, n, r, c, seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 6000 + seed)
    run_case(pp, n, r, keys, seed, opts=pp.options(rounds=2, host_loop=1, ctas_per_sm=1))


def test_tile_rounds_skip_tables_with_deletions(pp):
    """A table that saw a deletion may hold more keys in a cell than its count:
    the decode takes the binned rounds instead, with the same results."""
    n = (1 << 21) + 3
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.7, n), 71)
    run_case(pp, n, 3, keys, 71, deletes=keys[::7].copy())
    ghost = ppgen.distinct_keys(1000, 72)   # deletions of keys never inserted: negative counts
    gt = pp.IBLT(n, 3, 73, pp.options(rounds=2))
    ot = oracle.IBLT(n, 3, 73)
    gt.insert(_dev(keys))
    gt.delete(_dev(ghost))
    ot.insert(keys)
    ot.insert(ghost, sign=-1)
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    res = gt.decode(out)
    ores = ot.decode_rounds()
    assert res.rounds == ores["rounds"]
    assert res.recovered_per_round == [k.size for k in ores["keys"]]
    _assert_cells_equal(gt.cells(), ot)


def test_tile_rounds_residue_then_more_keys(pp):
    """Decode above the threshold (a residue is left), insert more keys, decode
    again: the record regions are sized from the counts at each decode's start."""
    n, r, seed = (1 << 21) + 7, 3, 81
    gt = pp.IBLT(n, r, seed)
    ot = oracle.IBLT(n, r, seed)
    k1 = ppgen.distinct_keys(ppgen.edges_from_c(0.9, n), 82)
    gt.insert(_dev(k1))
    ot.insert(k1)
    out = torch.zeros(k1.size * 2, dtype=torch.int64, device="cuda")
    res = gt.decode(out)
    ores = ot.decode_rounds()
    assert res.rounds == ores["rounds"] and res.residual_cells == ot.residual_cells() > 0
    _assert_cells_equal(gt.cells(), ot)
    k2 = ppgen.distinct_keys(ppgen.edges_from_c(0.05, n), 83)
    gt.insert(_dev(k2))
    ot.insert(k2)
    res = gt.decode(out)
    ores = ot.decode_rounds()
    assert res.rounds == ores["rounds"]
    assert res.recovered_per_round == [k.size for k in ores["keys"]]
    assert res.alive_cells_per_round == ores["cells_alive"]
    _assert_cells_equal(gt.cells(), ot)
    gt.close()


def test_tile_rounds_after_workspace_growth(pp):
    n, r = 3 * (1 << 19) + 5, 3
    gt = pp.IBLT(n, r, 5, pp.options(rounds=2))
    for m_frac in (0.1, 0.8, 0.75):
        keys = ppgen.distinct_keys(ppgen.edges_from_c(m_frac, n), int(m_frac * 100) + 7)
        gt.build(_dev(keys))
        out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
        res = gt.decode(out)
        ot = oracle.IBLT(n, r, 5)
        ot.insert(keys)
        ores = ot.decode_rounds()
        assert res.rounds == ores["rounds"]
        assert res.recovered_per_round == [k.size for k in ores["keys"]]
        _assert_cells_equal(gt.cells(), ot)


# ---- build + decode in one call: the build's tile pass finds F_1 -------------
def run_fused_case(pp, n, r, keys, seed, opts=None, max_rounds=None):
    """build_decode on the GPU against insert + decode_rounds in the oracle:
    per-round key sets, survivors and the residue, cell for cell."""
    gt = pp.IBLT(n, r, seed, opts)
    ot = oracle.IBLT(n, r, seed)
    ot.insert(keys)
    out = torch.zeros(max(1, keys.size), dtype=torch.int64, device="cuda")
    ores = ot.decode_rounds() if max_rounds is None else ot.decode_rounds(max_rounds=max_rounds)
    try:
        res = gt.build_decode(_dev(keys), out)
    except pp.PPError:
        _assert_cells_equal(gt.cells(), ot)       # what is left after the last completed round
        gt.close()
        raise
    assert res.rounds == ores["rounds"]
    got = out[: res.recovered].cpu().numpy().view(np.uint64)
    rounds = _split_rounds(got, res.recovered_per_round)
    assert len(rounds) == len(ores["keys"])
    for t, (a, b) in enumerate(zip(rounds, ores["keys"])):
        assert a.size == b.size and (a == np.sort(b)).all(), f"round {t + 1}"
    assert res.alive_cells_per_round == ores["cells_alive"]
    left = keys.size - np.cumsum([k.size for k in ores["keys"]])
    assert res.remaining_per_round == [int(x) for x in left]
    _assert_cells_equal(gt.cells(), ot)
    assert res.residual_cells == ot.residual_cells()
    gt.close()
    return res, ores


FUSED_CASES = [
    # n_cells, r, load c, seed: binned builds (forced on below 2^23 cells) into tile rounds
    (65541, 3, 0.75, 91),                   # one partial slab
    ((1 << 21) + 1, 4, 0.85, 92),           # above c*_{2,4}: a residue is left
    (3 * (1 << 21) + 17, 3, 0.75, 93),      # ragged last slab and tile
    ((1 << 22), 3, 0.90, 94),               # above c*_{2,3}
    ((1 << 22) + 5, 5, 0.60, 95),
]


@pytest.mark.parametrize("n,r,c,seed", FUSED_CASES, ids=[f"fused-n{n}-r{r}-c{c}" for n, r, c, _ in FUSED_CASES])
@pytest.mark.parametrize("host_loop", [0, 1], ids=["graph", "hostloop"])
def test_build_decode_parity(pp, n, r, c, seed, host_loop):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 9000 + seed)
    run_fused_case(pp, n, r, keys, seed, opts=pp.options(binned=1, rounds=2, host_loop=host_loop))


def test_build_decode_default_options_headline_shape(pp):
    """Default options at 2^23 cells: the slab-binned build and the tile rounds
    are both chosen, so the fused path runs."""
    n, r, seed = 1 << 23, 3, 96
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.75, n), 9096)
    res, _ = run_fused_case(pp, n, r, keys, seed)
    assert res.recovered == keys.size


@pytest.mark.parametrize("host_loop", [0, 1], ids=["graph", "hostloop"])
def test_build_decode_crowded_tile_is_rescanned(pp, host_loop):
    """Keys whose first cell falls in one 4096-cell tile push that tile's update
    list past its share (the mean tile's, with 15 % slack and 256 records), so
    the build cannot find F_1 there when it writes the tile out; the decode
    scans that tile itself and the results still match the oracle."""
    n, r, seed = 1 << 22, 3, 97
    base = ppgen.distinct_keys(ppgen.edges_from_c(0.6, n), 9097)
    cand = ppgen.distinct_keys(2_000_000, 9098)
    cand = np.setdiff1d(cand, base)
    first = oracle.key_cells(n, r, seed, cand)[:, 0].astype(np.int64)
    tile = 5
    crowd = cand[(first >> 12) == tile][:4000]
    keys = np.concatenate([base, crowd])
    cells = oracle.key_cells(n, r, seed, keys).astype(np.int64)
    per_tile = np.bincount((cells >> 12).ravel(), minlength=(n + 4095) >> 12)
    assert per_tile[tile] > 1.3 * per_tile.mean() + 256
    run_fused_case(pp, n, r, keys, seed, opts=pp.options(binned=1, rounds=2, host_loop=host_loop))


@pytest.mark.parametrize("host_loop", [0, 1], ids=["graph", "hostloop"])
@pytest.mark.parametrize("max_rounds", [1, 3])
def test_build_decode_round_limit(pp, host_loop, max_rounds):
    """Stopped by the round limit (after round 1: F_1's cells, emptied by the
    build, are put back), the table is the oracle's after that round."""
    n, r, seed = (1 << 21) + 3, 3, 98
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.80, n), 9099)
    opts = pp.options(binned=1, rounds=2, max_rounds=max_rounds, host_loop=host_loop)
    with pytest.raises(pp.PPError) as ei:
        run_fused_case(pp, n, r, keys, seed, opts=opts, max_rounds=max_rounds)
    assert ei.value.name == "PP_ERR_ROUND_LIMIT"


def test_build_decode_repeated_with_growth_and_plain_calls(pp):
    """build_decode with growing key counts (record buffers reallocated, the
    graphs rebuilt), mixed with plain build/insert/decode calls on the same
    table; also small tables and empty inputs, which take the unfused path."""
    n, r, seed = 3 * (1 << 20) + 11, 3, 99
    gt = pp.IBLT(n, r, seed, pp.options(binned=1, rounds=2))
    for i, c in enumerate((0.1, 0.8, 0.5, 0.0)):
        keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 9100 + i)
        out = torch.zeros(max(1, keys.size), dtype=torch.int64, device="cuda")
        res = gt.build_decode(_dev(keys), out)
        ot = oracle.IBLT(n, r, seed)
        ot.insert(keys)
        ores = ot.decode_rounds()
        assert res.rounds == ores["rounds"]
        assert res.recovered_per_round == [k.size for k in ores["keys"]]
        got = np.sort(out[: res.recovered].cpu().numpy().view(np.uint64))
        want = np.sort(np.concatenate(ores["keys"])) if ores["keys"] else np.zeros(0, np.uint64)
        assert (got == want).all()
        _assert_cells_equal(gt.cells(), ot)
        # a plain decode of more keys inserted on top uses the other graph
        more = ppgen.distinct_keys(ppgen.edges_from_c(0.05, n), 9200 + i)
        gt.insert(_dev(more))
        ot.insert(more)
        res = gt.decode(torch.zeros(more.size + keys.size, dtype=torch.int64, device="cuda"))
        ores = ot.decode_rounds()
        assert res.recovered_per_round == [k.size for k in ores["keys"]]
        _assert_cells_equal(gt.cells(), ot)
    gt.close()
    small = pp.IBLT(5000, 3, 7)
    keys = ppgen.distinct_keys(3000, 9300)
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    res, _ = run_fused_case(pp, 5000, 3, keys, 7)
    with pytest.raises(pp.PPError) as ei:
        small.build_decode(_dev(keys), out[:10])
    assert ei.value.name == "PP_ERR_CAPACITY"
    small.close()


def test_build_decode_slab_overflow_falls_back(pp):
    """Keys whose first cell falls in the first 2^21-cell slab overfill that
    slab's list: build_decode notices before the tile pass and builds with
    direct atomics, then decodes the plain way, with the oracle's results."""
    n, r, seed = 1 << 23, 3, 7
    cand = ppgen.distinct_keys(3_000_000, 8)
    first = oracle.key_cells(n, r, seed, cand)[:, 0]
    keys = cand[first < (1 << 21)]
    run_fused_case(pp, n, r, keys, seed)
