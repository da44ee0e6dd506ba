"""GPU parity of the batched decode: every table against the CPU oracle, and
against a plain per-table decode on the GPU (identical output)."""
import numpy as np
import pytest

import oracle
import ppgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ppb(ppeel_lib):
    import paper_1302_7014_b300 as pp
    import paper_1302_7014_b300.batch as batch
    return pp, batch


def _specs(count, seed, rs=(2, 3, 4, 5, 6), lo=5, hi=16, c_lo=0.3, c_hi=1.1):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(2 ** rng.uniform(lo, hi))
        r = int(rng.choice(rs))
        n = max(n, r)
        c = float(rng.uniform(c_lo, c_hi))
        specs.append((n, r, c, int(rng.integers(1, 2**62)), int(rng.integers(1, 2**62))))
    return specs


def run_batch(pp, batch_mod, specs, opts=None, out_slack=0):
    n_cells = [s[0] for s in specs]
    rs = [s[1] for s in specs]
    seeds = [s[3] for s in specs]
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    allk = np.concatenate(keys) if koff[-1] else np.zeros(1, np.uint64)
    b = batch_mod.Batch(n_cells, rs, seeds, opts)
    dk = torch.from_numpy(allk.view(np.int64)).cuda()
    b.insert(dk, koff)
    ooff = np.concatenate([[0], np.cumsum([k.size + out_slack for k in keys])]).astype(np.uint64)
    out = torch.full((max(1, int(ooff[-1])),), -1, dtype=torch.int64, device="cuda")
    res = b.decode(out, ooff)
    got = out.cpu().numpy().view(np.uint64)
    return b, keys, ooff, res, got


def check_against_oracle(specs, keys, ooff, res, got, b=None, cells_every=1):
    for i, (n, r, c, seed, _) in enumerate(specs):
        ot = oracle.IBLT(n, r, seed)
        ot.insert(keys[i])
        ores = ot.decode_rounds()
        assert res.rounds[i] == ores["rounds"], i
        assert res.recovered[i] == sum(k.size for k in ores["keys"]), i
        assert res.residual_cells[i] == ot.residual_cells(), i
        assert res.stats_complete[i]
        assert res.recovered_per_round[i] == [k.size for k in ores["keys"]], i
        region = got[int(ooff[i]): int(ooff[i]) + int(res.recovered[i])]
        ends = np.cumsum([0] + [k.size for k in ores["keys"]])
        for t, k in enumerate(ores["keys"]):
            assert (np.sort(region[ends[t]:ends[t + 1]]) == np.sort(k)).all(), (i, t)
        if b is not None and i % cells_every == 0:
            cells = b.cells(i)
            assert (cells["count"].astype(np.int64) == ot.count).all(), i
            assert (cells["key_xor"] == ot.keyx).all() and (cells["chk_xor"] == ot.chkx).all(), i


def test_mixed_ranks(ppb):
    pp, bm = ppb
    specs = _specs(60, 1)
    b, keys, ooff, res, got = run_batch(pp, bm, specs)
    check_against_oracle(specs, keys, ooff, res, got, b)


@pytest.mark.parametrize("r", [3, 4])
def test_uniform_rank(ppb, r):
    pp, bm = ppb
    specs = _specs(40, 10 + r, rs=(r,), lo=8, hi=17, c_lo=0.5, c_hi=0.95)
    b, keys, ooff, res, got = run_batch(pp, bm, specs, out_slack=3)
    check_against_oracle(specs, keys, ooff, res, got, b, cells_every=4)


def test_host_loop_and_small_grid(ppb):
    pp, bm = ppb
    specs = _specs(30, 3)
    for opts in (pp.options(host_loop=1), pp.options(ctas_per_sm=1)):
        b, keys, ooff, res, got = run_batch(pp, bm, specs, opts)
        check_against_oracle(specs, keys, ooff, res, got)


def test_batched_workload_prefix_matches_plain(ppb):
    # the first 300 tables of the 4096-table recipe: batch == plain per-table decode
    pp, bm = ppb
    tabs = ppgen.batch_tables(4096)[:300]
    specs = [(t.n_cells, t.r, t.c, t.table_seed, t.key_seed) for t in tabs]
    b, keys, ooff, res, got = run_batch(pp, bm, specs)
    for i, (n, r, c, seed, _) in enumerate(specs):
        t = pp.IBLT(n, r, seed)
        t.insert(torch.from_numpy(keys[i].view(np.int64)).cuda())
        out = torch.zeros(max(1, keys[i].size), dtype=torch.int64, device="cuda")
        pr = t.decode(out)
        assert pr.rounds == res.rounds[i] and pr.recovered == res.recovered[i]
        assert pr.recovered_per_round == res.recovered_per_round[i]
        assert pr.residual_cells == res.residual_cells[i]
        mine = got[int(ooff[i]): int(ooff[i]) + pr.recovered]
        theirs = out[: pr.recovered].cpu().numpy().view(np.uint64)
        ends = np.cumsum([0] + pr.recovered_per_round)
        for a0, a1 in zip(ends[:-1], ends[1:]):
            assert (np.sort(mine[a0:a1]) == np.sort(theirs[a0:a1])).all()
        t.close()
    # and a sample against the oracle
    for i in range(0, 300, 7):
        n, r, c, seed, _ = specs[i]
        ot = oracle.IBLT(n, r, seed)
        ot.insert(keys[i])
        ores = ot.decode_rounds()
        assert res.recovered_per_round[i] == [k.size for k in ores["keys"]]


def test_capacity_and_reuse(ppb):
    pp, bm = ppb
    specs = _specs(8, 5, lo=8, hi=12)
    b, keys, ooff, res, got = run_batch(pp, bm, specs)
    # re-insert, decode into a different buffer with one table short of room
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    b.clear()
    b.insert(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff)
    short = ooff.copy()
    short[3:] -= 1
    out2 = torch.zeros(int(ooff[-1]), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError) as ei:
        b.decode(out2, short)
    assert ei.value.name == "PP_ERR_CAPACITY"
    res2 = b.decode(out2, ooff)   # a new output buffer: the graph is rebuilt
    got2 = out2.cpu().numpy().view(np.uint64)
    check_against_oracle(specs, keys, ooff, res2, got2)


def test_empty_tables_in_batch(ppb):
    pp, bm = ppb
    specs = [(100, 3, 0.0, 1, 2), (257, 4, 0.5, 3, 4), (64, 3, 0.0, 5, 6)]
    b, keys, ooff, res, got = run_batch(pp, bm, specs)
    check_against_oracle(specs, keys, ooff, res, got, b)
    assert res.rounds[0] == 0 and res.rounds[2] == 0


@pytest.mark.parametrize("rs,rounds", [((3, 4), 1), ((2, 3, 5, 6), 1), ((3, 4), 2), ((2, 3, 5, 6), 2)],
                         ids=["r3-4-binned", "r2-6-binned", "r3-4-tiles", "r2-6-tiles"])
def test_binned_batch_build_and_rounds(ppb, rs, rounds):
    """Slab-binned build (forced on) and binned or tile rounds over the arena, mixed ranks."""
    pp, bm = ppb
    specs = _specs(50, 77 + len(rs), rs=rs, lo=10, hi=17, c_lo=0.5, c_hi=0.95)
    n_cells = [s[0] for s in specs]
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    dk = torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda()
    b = bm.Batch(n_cells, [s[1] for s in specs], [s[3] for s in specs], pp.options(binned=1, rounds=rounds))
    b.insert(torch.from_numpy(ppgen.distinct_keys(int(koff[-1]), 3).view(np.int64)).cuda(), koff)  # junk
    b.build(dk, koff)                       # must wipe the junk
    for i in range(0, len(specs), 5):
        ot = oracle.IBLT(specs[i][0], specs[i][1], specs[i][3])
        ot.insert(keys[i])
        cells = b.cells(i)
        assert (cells["count"].astype(np.int64) == ot.count).all()
        assert (cells["key_xor"] == ot.keyx).all() and (cells["chk_xor"] == ot.chkx).all()
    out = torch.full((int(koff[-1]),), -1, dtype=torch.int64, device="cuda")
    res = b.decode(out, koff)
    check_against_oracle(specs, keys, koff, res, out.cpu().numpy().view(np.uint64), b, cells_every=3)
    # incremental insert + delete through the binned path
    b.clear()
    b.insert(dk, koff)
    dele = [k[::4] for k in keys]
    doff = np.concatenate([[0], np.cumsum([d.size for d in dele])]).astype(np.uint64)
    b.delete(torch.from_numpy(np.concatenate(dele).view(np.int64)).cuda(), doff)
    for i in range(0, len(specs), 7):
        ot = oracle.IBLT(specs[i][0], specs[i][1], specs[i][3])
        ot.insert(keys[i])
        ot.insert(dele[i], sign=-1)
        cells = b.cells(i)
        assert (cells["count"].astype(np.int64) == ot.count).all()
        assert (cells["key_xor"] == ot.keyx).all()


@pytest.mark.parametrize("rs,big,rounds", [((3, 4), False, 1), ((2, 5, 6), False, 1), ((3, 4), True, 1),
                                           ((3, 4), False, 0), ((2, 5, 6), True, 0)],
                         ids=["keys-r3-4", "keys-r2-6", "slab-lists", "keys-r3-4-tiles", "slab-lists-r2-6-tiles"])
def test_binned_batch_build_across_slabs(ppb, rs, big, rounds):
    """Tables spread over several 2^21-cell slabs, some straddling two.  Such
    a batch is built with each slab's keys hashed inside the tile pass; with
    one table larger than a slab it takes the slab-list build instead.  Build,
    insert and delete cell for cell, and the decode, against the oracle."""
    pp, bm = ppb
    specs = _specs(24, 131 + len(rs), rs=rs, lo=17, hi=20.6, c_lo=0.5, c_hi=0.9)
    if big:
        s5 = specs[5]
        specs[5] = ((1 << 21) + 4099, 3, 0.7, s5[3], s5[4])
    n_cells = [s[0] for s in specs]
    assert sum(n_cells) > 4 * (1 << 21)
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    dk = torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda()
    b = bm.Batch(n_cells, [s[1] for s in specs], [s[3] for s in specs], pp.options(binned=1, rounds=rounds))
    b.insert(torch.from_numpy(ppgen.distinct_keys(int(koff[-1]), 5).view(np.int64)).cuda(), koff)  # junk
    b.build(dk, koff)                       # must wipe the junk
    ots = []
    for i, s in enumerate(specs):
        ot = oracle.IBLT(s[0], s[1], s[3])
        ot.insert(keys[i])
        ots.append(ot)
        cells = b.cells(i)
        assert (cells["count"].astype(np.int64) == ot.count).all(), i
        assert (cells["key_xor"] == ot.keyx).all() and (cells["chk_xor"] == ot.chkx).all(), i
    out = torch.full((int(koff[-1]),), -1, dtype=torch.int64, device="cuda")
    res = b.decode(out, koff)
    check_against_oracle(specs, keys, koff, res, out.cpu().numpy().view(np.uint64), b, cells_every=4)
    # incremental insert + delete through the same path
    b.clear()
    b.insert(dk, koff)
    dele = [k[::5] for k in keys]
    doff = np.concatenate([[0], np.cumsum([d.size for d in dele])]).astype(np.uint64)
    b.delete(torch.from_numpy(np.concatenate(dele).view(np.int64)).cuda(), doff)
    for i in range(0, len(specs), 3):
        ots[i].insert(dele[i], sign=-1)
        cells = b.cells(i)
        assert (cells["count"].astype(np.int64) == ots[i].count).all(), i
        assert (cells["key_xor"] == ots[i].keyx).all() and (cells["chk_xor"] == ots[i].chkx).all(), i


def test_binned_batch_decode_after_deletions(ppb):
    """Residue counted by the scan (no shortcut once keys were deleted)."""
    pp, bm = ppb
    specs = _specs(30, 91, rs=(3, 4), lo=10, hi=15, c_lo=0.6, c_hi=1.0)
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs], pp.options(binned=1))
    b.insert(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff)
    dele = [k[::3] for k in keys]
    doff = np.concatenate([[0], np.cumsum([d.size for d in dele])]).astype(np.uint64)
    b.delete(torch.from_numpy(np.concatenate(dele).view(np.int64)).cuda(), doff)
    left = [np.setdiff1d(k, d) for k, d in zip(keys, dele)]
    ooff = np.concatenate([[0], np.cumsum([x.size for x in left])]).astype(np.uint64)
    out = torch.full((int(ooff[-1]),), -1, dtype=torch.int64, device="cuda")
    res = b.decode(out, ooff)
    got = out.cpu().numpy().view(np.uint64)
    for i, s in enumerate(specs):
        ot = oracle.IBLT(s[0], s[1], s[3])
        ot.insert(keys[i])
        ot.insert(dele[i], sign=-1)
        ores = ot.decode_rounds()
        assert res.rounds[i] == ores["rounds"]
        assert res.residual_cells[i] == ot.residual_cells()
        region = np.sort(got[int(ooff[i]): int(ooff[i]) + int(res.recovered[i])])
        want = np.sort(np.concatenate(ores["keys"])) if ores["keys"] else np.zeros(0, np.uint64)
        assert (region == want).all()


@pytest.mark.parametrize("binned", [1, 2])
def test_batch_deleting_keys_never_inserted(ppb, binned):
    """Negative counts in every table: the per-table residue is the number of
    cells with a non-zero count, as in the oracle, with either round kind."""
    pp, bm = ppb
    specs = _specs(20, 93 + binned, rs=(3, 4), lo=10, hi=15, c_lo=0.5, c_hi=0.9)
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    ghost = [ppgen.distinct_keys(max(1, s[0] // 20), 1000 + i) for i, s in enumerate(specs)]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    goff = np.concatenate([[0], np.cumsum([g.size for g in ghost])]).astype(np.uint64)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs],
                 pp.options(binned=binned))
    b.insert(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff)
    b.delete(torch.from_numpy(np.concatenate(ghost).view(np.int64)).cuda(), goff)
    out = torch.full((int(koff[-1]),), -1, dtype=torch.int64, device="cuda")
    res = b.decode(out, koff)
    for i, s in enumerate(specs):
        ot = oracle.IBLT(s[0], s[1], s[3])
        ot.insert(keys[i])
        ot.insert(ghost[i], sign=-1)
        ores = ot.decode_rounds()
        assert res.rounds[i] == ores["rounds"], i
        assert res.recovered[i] == sum(k.size for k in ores["keys"]), i
        assert res.residual_cells[i] == ot.residual_cells(), i


# ---- tile rounds over the arena ---------------------------------------------
@pytest.mark.parametrize("opts", [dict(rounds=2), dict(rounds=2, host_loop=1), dict(rounds=2, ctas_per_sm=1)],
                         ids=["graph", "hostloop", "small-grid"])
def test_tile_rounds_mixed_ranks(ppb, opts):
    """Tile rounds (forced on for a small arena) with tables of r = 2..6 sharing
    tiles: every table against the oracle, cell for cell."""
    pp, bm = ppb
    specs = _specs(60, 201, lo=5, hi=15, c_lo=0.3, c_hi=1.05)
    b, keys, ooff, res, got = run_batch(pp, bm, specs, pp.options(**opts), out_slack=2)
    check_against_oracle(specs, keys, ooff, res, got, b)


@pytest.mark.parametrize("r", [3, 4])
def test_tile_rounds_uniform_rank(ppb, r):
    pp, bm = ppb
    specs = _specs(40, 220 + r, rs=(r,), lo=8, hi=17, c_lo=0.5, c_hi=0.95)
    b, keys, ooff, res, got = run_batch(pp, bm, specs, pp.options(rounds=2))
    check_against_oracle(specs, keys, ooff, res, got, b, cells_every=3)


@pytest.mark.parametrize("host_loop", [0, 1])
def test_tile_rounds_round_limit(ppb, host_loop):
    """A batched decode in tile rounds stopped by the round limit leaves every
    table as the oracle's after that round (the pending frontier's cells put
    back), with the per-table statistics of the rounds that ran."""
    pp, bm = ppb
    specs = _specs(16, 231, rs=(3, 4), lo=11, hi=15, c_lo=0.7, c_hi=0.8)
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs],
                 pp.options(max_rounds=3, rounds=2, host_loop=host_loop))
    b.insert(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff)
    out = torch.full((int(koff[-1]),), -1, dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError) as ei:
        b.decode(out, koff)
    assert ei.value.name == "PP_ERR_ROUND_LIMIT"
    for i, s in enumerate(specs):
        ot = oracle.IBLT(s[0], s[1], s[3])
        ot.insert(keys[i])
        ot.decode_rounds(max_rounds=3)
        cells = b.cells(i)
        assert (cells["count"].astype(np.int64) == ot.count).all(), i
        assert (cells["key_xor"] == ot.keyx).all() and (cells["chk_xor"] == ot.chkx).all(), i


def test_tile_rounds_fall_back_after_deletions(ppb):
    """A batch that saw a deletion decodes in binned rounds even when tile
    rounds are asked for, and still matches the oracle."""
    pp, bm = ppb
    specs = _specs(20, 241, rs=(3, 4), lo=10, hi=15, c_lo=0.5, c_hi=0.9)
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs], pp.options(rounds=2))
    b.insert(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff)
    dele = [k[::4] for k in keys]
    doff = np.concatenate([[0], np.cumsum([d.size for d in dele])]).astype(np.uint64)
    b.delete(torch.from_numpy(np.concatenate(dele).view(np.int64)).cuda(), doff)
    left = [np.setdiff1d(k, d) for k, d in zip(keys, dele)]
    ooff = np.concatenate([[0], np.cumsum([x.size for x in left])]).astype(np.uint64)
    out = torch.full((max(1, int(ooff[-1])),), -1, dtype=torch.int64, device="cuda")
    res = b.decode(out, ooff)
    got = out.cpu().numpy().view(np.uint64)
    for i, s in enumerate(specs):
        ot = oracle.IBLT(s[0], s[1], s[3])
        ot.insert(keys[i])
        ot.insert(dele[i], sign=-1)
        ores = ot.decode_rounds()
        assert res.rounds[i] == ores["rounds"], i
        assert res.residual_cells[i] == ot.residual_cells(), i
        region = np.sort(got[int(ooff[i]): int(ooff[i]) + int(res.recovered[i])])
        want = np.sort(np.concatenate(ores["keys"])) if ores["keys"] else np.zeros(0, np.uint64)
        assert (region == want).all(), i


def test_tile_rounds_decode_twice_and_reuse(ppb):
    """Tile rounds over the arena: a second decode finds nothing left (the
    residue is a 2-core), and the batch cleared and refilled with other keys
    decodes them exactly (the graph and buffers are reused or rebuilt)."""
    pp, bm = ppb
    specs = _specs(24, 251, rs=(3, 4), lo=10, hi=15, c_lo=0.6, c_hi=1.0)
    b, keys, ooff, res, got = run_batch(pp, bm, specs, pp.options(rounds=2))
    check_against_oracle(specs, keys, ooff, res, got, b)
    out = torch.full((max(1, int(ooff[-1])),), -1, dtype=torch.int64, device="cuda")
    res2 = b.decode(out, ooff)
    for i in range(len(specs)):
        assert res2.rounds[i] == 0 and res2.recovered[i] == 0, i
        assert res2.residual_cells[i] == res.residual_cells[i], i
    specs2 = [(s[0], s[1], s[2] * 0.8, s[3], s[4] + 1) for s in specs]
    keys2 = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs2]
    koff2 = np.concatenate([[0], np.cumsum([k.size for k in keys2])]).astype(np.uint64)
    b.clear()
    b.insert(torch.from_numpy(np.concatenate(keys2).view(np.int64)).cuda(), koff2)
    out2 = torch.full((max(1, int(koff2[-1])),), -1, dtype=torch.int64, device="cuda")
    res3 = b.decode(out2, koff2)
    check_against_oracle(specs2, keys2, koff2, res3, out2.cpu().numpy().view(np.uint64), b, cells_every=2)


# ---- build + decode in one call: the build's tile write-out finds F_1 --------
def run_fused_batch(pp, bm, specs, opts, keys=None, max_rounds=None):
    """Batch.build_decode against the oracle, table by table (keys, rounds,
    survivors, residue cell for cell)."""
    if keys is None:
        keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs], opts)
    # junk first: the build must wipe it and the decode must not see it
    b.insert(torch.from_numpy(ppgen.distinct_keys(int(koff[-1]), 5).view(np.int64)).cuda(), koff)
    out = torch.full((max(1, int(koff[-1])),), -1, dtype=torch.int64, device="cuda")
    dk = torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda()
    if max_rounds is None:
        res = b.build_decode(dk, koff, out, koff)
        check_against_oracle(specs, keys, koff, res, out.cpu().numpy().view(np.uint64), b)
    else:
        with pytest.raises(pp.PPError) as ei:
            b.build_decode(dk, koff, out, koff)
        assert ei.value.name == "PP_ERR_ROUND_LIMIT"
        for i, s in enumerate(specs):
            ot = oracle.IBLT(s[0], s[1], s[3])
            ot.insert(keys[i])
            ot.decode_rounds(max_rounds=max_rounds)
            cells = b.cells(i)
            assert (cells["count"].astype(np.int64) == ot.count).all(), i
            assert (cells["key_xor"] == ot.keyx).all() and (cells["chk_xor"] == ot.chkx).all(), i
    return b, keys, koff


@pytest.mark.parametrize("rs,opts", [((3,), dict(binned=1, rounds=2)), ((3, 4), dict(binned=1, rounds=2)),
                                     ((2, 3, 5, 6), dict(binned=1, rounds=2)),
                                     ((3, 4), dict(binned=1, rounds=2, host_loop=1)),
                                     ((3,), dict(binned=1, rounds=2, ctas_per_sm=1))],
                         ids=["r3", "r3-4", "r2-6", "r3-4-hostloop", "r3-small-grid"])
def test_batch_build_decode_parity(ppb, rs, opts):
    """Tables over several 2^21-cell slabs, some straddling two: the keys'
    tile pass finds F_1 as it writes each tile out and the tile rounds start
    from it.  Every table against the oracle."""
    pp, bm = ppb
    specs = _specs(24, 301 + len(rs), rs=rs, lo=15, hi=20.6, c_lo=0.5, c_hi=0.95)
    assert sum(s[0] for s in specs) > 2 * (1 << 21)
    # loads near the threshold take hundreds of rounds: keep every round's count
    run_fused_batch(pp, bm, specs, pp.options(stats_rounds=4096, **opts))


@pytest.mark.parametrize("host_loop", [0, 1], ids=["graph", "hostloop"])
@pytest.mark.parametrize("max_rounds", [1, 3])
def test_batch_build_decode_round_limit(ppb, host_loop, max_rounds):
    pp, bm = ppb
    specs = _specs(16, 331, rs=(3, 4), lo=15, hi=19, c_lo=0.7, c_hi=0.8)
    run_fused_batch(pp, bm, specs, pp.options(binned=1, rounds=2, max_rounds=max_rounds, host_loop=host_loop),
                    max_rounds=max_rounds)


def test_batch_build_decode_crowded_tile_is_rescanned(ppb):
    """One table's keys crowd the first 4096-cell tile of the arena past its
    list's share, so the build leaves that tile to the decode's rescan."""
    pp, bm = ppb
    specs = _specs(12, 341, rs=(3,), lo=16, hi=19, c_lo=0.6, c_hi=0.7)
    n0 = 1 << 20
    specs[0] = (n0, 3, 0.6, specs[0][3], specs[0][4])
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    cand = np.setdiff1d(ppgen.distinct_keys(2_000_000, 342), keys[0])
    first = oracle.key_cells(n0, 3, specs[0][3], cand)[:, 0].astype(np.int64)
    keys[0] = np.concatenate([keys[0], cand[first < 4096][:3000]])
    cells = oracle.key_cells(n0, 3, specs[0][3], keys[0]).astype(np.int64)
    per_tile = np.bincount((cells >> 12).ravel())
    assert per_tile[0] > 1.3 * per_tile[1:].mean() + 256
    for hl in (0, 1):
        run_fused_batch(pp, bm, specs, pp.options(binned=1, rounds=2, host_loop=hl, stats_rounds=4096), keys=keys)


def test_batch_build_decode_unfused_cases(ppb):
    """Where the build cannot find F_1 (a table larger than a slab, or a batch
    built with direct atomics) the call builds and decodes one after the other,
    with the same results; repeated calls and a plain decode after more
    inserts stay right."""
    pp, bm = ppb
    specs = _specs(10, 351, rs=(3, 4), lo=12, hi=17, c_lo=0.5, c_hi=0.9)
    specs[3] = ((1 << 21) + 4099, 3, 0.7, specs[3][3], specs[3][4])
    run_fused_batch(pp, bm, specs, pp.options(binned=1, rounds=2, stats_rounds=4096))  # slab lists
    small = _specs(30, 352, rs=(3, 4), lo=6, hi=12, c_lo=0.5, c_hi=0.9)
    b, keys, koff = run_fused_batch(pp, bm, small, pp.options(stats_rounds=4096))  # small arena: direct atomics
    for rep in range(2):                                                    # again, and on top of a decode
        out = torch.full((int(koff[-1]),), -1, dtype=torch.int64, device="cuda")
        res = b.build_decode(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff, out, koff)
        check_against_oracle(small, keys, koff, res, out.cpu().numpy().view(np.uint64), b)
    with pytest.raises(pp.PPError) as ei:
        short = koff.copy()
        short[1:] -= 1
        short[0] = 0
        b.build_decode(torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda(), koff, out,
                       np.maximum.accumulate(short))
    assert ei.value.name == "PP_ERR_CAPACITY"
