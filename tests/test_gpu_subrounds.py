"""GPU parity: peeling and IBLT recovery with sub-tables (App. B) against the
CPU oracle.

Exact comparisons: every vertex's and edge's removal sub-round, the per
sub-round survivor counts and the sub-round count S (k-core); every
sub-round's recovered key set, S, the residue left in the table bit for bit
(IBLT).  Sizes span several chunks with ragged tails; the full-size cases
check properties that hold at any size against the full-round path.
"""
import numpy as np
import pytest

import oracle
import ppgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pp(ppeel_lib):
    import paper_1302_7014_b300 as pp
    return pp


def _offsets(n, p):
    return [int(x) for x in oracle.part_offsets(n, p)]


def _dev_edges(edges, r):
    if edges.shape[0] == 0:
        return torch.zeros((0, r), dtype=torch.int32, device="cuda")
    return torch.from_numpy(np.ascontiguousarray(edges, dtype=np.uint32).view(np.int32)).cuda()


def gpu_sub(pp, n, r, k, edges, off, opts=None):
    m = edges.shape[0]
    vr = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    er = torch.full((max(m, 1),), -7, dtype=torch.int32, device="cuda")
    res = pp.peel_kcore_subrounds(n, r, k, _dev_edges(edges, r), off, vr[:n] if n else None,
                                  er[:m] if m else None, opts, round_cap=1 << 16)
    return res, vr[:n].cpu().numpy(), er[:m].cpu().numpy()


def check_kcore(pp, n, k, edges, off, opts=None):
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    r = edges.shape[1]
    res, vr, er = gpu_sub(pp, n, r, k, edges, off, opts)
    o = oracle.kcore_subrounds(n, k, edges, off)
    assert res.rounds == o["subrounds"]
    assert (vr == o["vround"]).all()
    assert (er == o["eround"]).all()
    assert res.vertices_left == o["s"] and res.edges_left == o["m"]
    assert res.core_vertices == int((o["vround"] == 0).sum())
    assert res.core_edges == int((o["eround"] == 0).sum())
    return res


def test_kcore_hand_worked(pp):
    check_kcore(pp, 4, 2, np.array([[0, 2], [2, 1], [1, 3]]), [0, 2, 4])
    res = check_kcore(pp, 5, 2, np.array([[0, 1, 4], [2, 3, 4]]), [0, 2, 2, 5])
    assert res.rounds == 3 and res.vertices_left == [3, 3, 0]


def test_kcore_random_small(pp):
    rng = np.random.default_rng(21)
    for trial in range(40):
        n = int(rng.integers(1, 400))
        r = int(rng.integers(2, 6))
        m = int(rng.integers(0, 3 * n))
        k = int(rng.integers(1, 4))
        p = int(rng.integers(1, 7))
        off = [0] + sorted(int(x) for x in rng.integers(0, n + 1, size=p - 1)) + [n]
        e = rng.integers(0, n, size=(m, r), dtype=np.uint32)
        check_kcore(pp, n, k, e, off)


@pytest.mark.parametrize("n,r,c,k,seed", [
    (3 * 1024 + 5, 3, 0.75, 2, 1),
    (20000, 4, 0.70, 2, 2),
    (20000, 4, 0.85, 2, 3),      # above c*_{2,4}: a 2-core is left
    (50001, 3, 1.2, 3, 4),       # k = 3
    (65536 + 77, 2, 0.45, 2, 5),  # r = 2 (a graph)
    (30000, 5, 0.6, 2, 6),
])
def test_kcore_partitioned(pp, n, r, c, k, seed):
    e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(c, n), seed)
    check_kcore(pp, n, k, e, _offsets(n, r))


def test_kcore_one_part_equals_full_rounds(pp):
    n, r = 40000, 4
    e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(0.74, n), 9)
    a = check_kcore(pp, n, 2, e, [0, n])
    d = _dev_edges(e, r)
    b = pp.peel_kcore(n, r, 2, d)
    assert a.rounds == b.rounds and a.vertices_left == b.vertices_left and a.edges_left == b.edges_left


def test_kcore_2e22_exact(pp):
    n, r = 1 << 22, 4
    e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(0.78, n), 3)
    check_kcore(pp, n, 2, e, _offsets(n, r))


def test_kcore_full_size_properties(pp):
    # n = 2^25, r = 4 at two densities of the k-core sweep: the sub-round
    # process reaches the same core as full rounds (the core is unique), in at
    # most r times as many sub-rounds, never leaving more vertices after round
    # i's last sub-round than full round i does
    n, r = 1 << 25, 4
    off = _offsets(n, r)
    for c in (0.76, 0.80):
        e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(c, n), 3)
        d = _dev_edges(e, r)
        del e
        vr_a = torch.empty(n, dtype=torch.int32, device="cuda")
        vr_b = torch.empty(n, dtype=torch.int32, device="cuda")
        a = pp.peel_kcore(n, r, 2, d, vr_a)
        b = pp.peel_kcore_subrounds(n, r, 2, d, off, vr_b, round_cap=1 << 16)
        assert torch.equal(vr_a == 0, vr_b == 0)
        assert a.core_vertices == b.core_vertices and a.core_edges == b.core_edges
        assert b.rounds <= r * a.rounds
        for i in range(1, a.rounds + 1):
            left = b.vertices_left[r * i - 1] if r * i <= b.rounds else b.core_vertices
            assert left <= a.vertices_left[i - 1], i
        del d, vr_a, vr_b
        torch.cuda.empty_cache()


@pytest.mark.parametrize("hub_deg", [65535, 65536])
def test_kcore_high_degree_vertex(pp, hub_deg):
    """A vertex of degree 65535 (16-bit counters) and 65536 (32-bit recount)."""
    n, r = 50000, 3
    rng = np.random.default_rng(hub_deg)
    e = rng.integers(2, n, size=(hub_deg, r), dtype=np.uint64).astype(np.uint32)
    e[:, 0] = 1
    filler = (ppgen.uniform_edges(n - 2, r, 20000, 5).astype(np.uint64) + 2).astype(np.uint32)
    edges = np.concatenate([e, filler])
    assert int((edges == 1).sum()) == hub_deg
    check_kcore(pp, n, 2, edges, _offsets(n, 3))


def test_kcore_round_limit(pp):
    n, r = 20000, 4
    e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(0.7, n), 5)
    with pytest.raises(pp.PPError) as ei:
        gpu_sub(pp, n, r, 2, e, _offsets(n, r), pp.options(max_rounds=3))
    assert ei.value.name == "PP_ERR_ROUND_LIMIT"


def test_kcore_empty_and_edgeless(pp):
    res, vr, _ = gpu_sub(pp, 10, 3, 2, np.zeros((0, 3), np.uint32), [0, 3, 7, 10])
    # every vertex has degree 0 < 2: each part goes in its own sub-round
    assert res.rounds == 3 and list(vr) == [1] * 3 + [2] * 4 + [3] * 3
    assert res.vertices_left == [7, 3, 0]


def test_kcore_bad_parts(pp):
    e = np.array([[0, 1, 2]], np.uint32)
    for off in ([0, 2], [1, 3], [0, 2, 1, 3]):
        with pytest.raises(pp.PPError) as ei:
            gpu_sub(pp, 3, 3, 2, e, off)
        assert ei.value.name == "PP_ERR_INVALID_ARG"


# ----------------------------------------------------------------------------
# IBLT
# ----------------------------------------------------------------------------
def _dev(keys):
    return torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()


def _assert_cells_equal(cells, ot):
    assert (cells["count"].astype(np.int64) == ot.count).all()
    assert (cells["key_xor"] == ot.keyx).all()
    assert (cells["chk_xor"] == ot.chkx).all()


def run_iblt(pp, n, r, keys, seed, opts=None, deletes=None, max_sub=None):
    gt = pp.IBLT(n, r, seed, opts)
    ot = oracle.IBLT(n, r, seed)
    if len(keys):
        gt.insert(_dev(keys))
    ot.insert(keys)
    if deletes is not None and len(deletes):
        gt.delete(_dev(deletes))
        ot.insert(deletes, sign=-1)
    items = len(keys) - (0 if deletes is None else len(deletes))
    # keys deleted without being inserted leave count -1 cells; the inserted
    # keys can all come out, so the output holds every inserted key
    out = torch.zeros(max(1, len(keys)), dtype=torch.int64, device="cuda")
    res = gt.decode_subrounds(out, round_cap=1 << 16)
    ores = ot.decode_subrounds() if max_sub is None else ot.decode_subrounds(max_subrounds=max_sub)
    assert res.rounds == ores["subrounds"]
    got = out[: res.recovered].cpu().numpy().view(np.uint64)
    ends = np.cumsum([0] + list(res.recovered_per_round))
    assert ends[-1] == res.recovered
    for s, want in enumerate(ores["keys"]):
        a = np.sort(got[ends[s]:ends[s + 1]])
        assert a.size == want.size and (a == want).all(), f"sub-round {s + 1}"
    left = np.maximum(items - np.cumsum([k.size for k in ores["keys"]]), 0)
    assert res.remaining_per_round == [int(x) for x in left]
    _assert_cells_equal(gt.cells(), ot)
    assert res.residual_cells == ot.residual_cells()
    gt.close()
    return res, ores


@pytest.mark.parametrize("n,r,c,seed", [
    (1000, 3, 0.70, 1),
    (3 * 1024 + 17, 3, 0.75, 2),
    (50021, 3, 0.80, 3),
    (65536, 4, 0.70, 4),
    (40000, 3, 0.90, 5),    # above c*_{2,3}: a residue stays
    (30011, 5, 0.60, 6),    # generic kernel
    (20000, 2, 0.40, 7),
])
def test_iblt_subrounds(pp, n, r, c, seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 100 + seed)
    run_iblt(pp, n, r, keys, seed)


def test_iblt_subrounds_with_deletions(pp):
    n, r = 30000, 3
    keys = ppgen.distinct_keys(26000, 8)
    # delete a third of the keys, plus some that were never inserted
    dels = np.concatenate([keys[::3], ppgen.distinct_keys(500, 9)])
    run_iblt(pp, n, r, keys, 11, deletes=dels)


@pytest.mark.parametrize("n,r,c,binned,host_loop", [
    (50021, 3, 0.78, 1, 0),     # binned sub-rounds forced on a small table
    (50021, 3, 0.78, 1, 1),
    (1 << 21, 4, 0.72, 0, 1),   # binned by size, rounds driven from the host
    (1 << 22, 3, 0.75, 2, 0),   # plain kernels forced on a large table
])
def test_iblt_subrounds_both_kernel_paths(pp, n, r, c, binned, host_loop):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 30 + r)
    run_iblt(pp, n, r, keys, 31, opts=pp.options(binned=binned, host_loop=host_loop))


def test_iblt_subrounds_binned_table_size(pp):
    # 2^22 cells: the size where the full-round decode switches to binned rounds
    n, r = 1 << 22, 3
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.75, n), 12)
    run_iblt(pp, n, r, keys, 13)


def test_iblt_subrounds_empty_table(pp):
    gt = pp.IBLT(5000, 3, 1)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    res = gt.decode_subrounds(out)
    assert res.rounds == 0 and res.recovered == 0 and res.residual_cells == 0


def test_iblt_subrounds_round_limit(pp):
    n, r = 20000, 3
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.75, n), 14)
    gt = pp.IBLT(n, r, 15, pp.options(max_rounds=4))
    gt.insert(_dev(keys))
    out = torch.zeros(len(keys), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError) as ei:
        gt.decode_subrounds(out)
    assert ei.value.name == "PP_ERR_ROUND_LIMIT"


def test_iblt_subrounds_host_loop_matches_graph(pp):
    n, r = 100003, 3
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.78, n), 16)
    res_a, _ = run_iblt(pp, n, r, keys, 17)
    res_b, _ = run_iblt(pp, n, r, keys, 17, opts=pp.options(host_loop=1))
    assert res_a.recovered_per_round == res_b.recovered_per_round


def test_iblt_subrounds_twice_on_one_handle(pp):
    # the sub-round graph is built once per handle and reused
    n, r = 50000, 3
    gt = pp.IBLT(n, r, 18)
    for rep in range(2):
        keys = ppgen.distinct_keys(ppgen.edges_from_c(0.7, n), 19 + rep)
        gt.build(_dev(keys))
        out = torch.zeros(len(keys), dtype=torch.int64, device="cuda")
        res = gt.decode_subrounds(out)
        got = np.sort(out[: res.recovered].cpu().numpy().view(np.uint64))
        assert (got == np.sort(keys)).all() and res.residual_cells == 0


def test_iblt_subrounds_headline_size(pp):
    # the 2^26-cell headline table: every key comes out once, the residue is
    # empty, and the full-round decode of the same table agrees
    n, r = 1 << 26, 3
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.75, n), 2)
    dk = _dev(keys)
    out = torch.zeros(len(keys), dtype=torch.int64, device="cuda")
    gt = pp.IBLT(n, r, 0x13027014)
    gt.build(dk)
    res = gt.decode_subrounds(out, round_cap=1 << 12)
    got = np.sort(out.cpu().numpy().view(np.uint64))
    assert res.recovered == len(keys) and res.residual_cells == 0
    assert (got == np.sort(keys)).all()
    assert sum(res.recovered_per_round) == len(keys)
    sub_rounds = res.rounds
    gt.build(dk)
    full = gt.decode(out)
    assert full.recovered == len(keys)
    # App. B: at most r sub-rounds per round
    assert sub_rounds <= r * full.rounds
    gt.close()
