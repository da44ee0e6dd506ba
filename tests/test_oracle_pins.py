"""Pins for the CPU oracle, each against something other than the oracle itself.

* k-core: brute force over all vertex subsets (Sec. 1: the k-core is the
  maximal subgraph of minimum degree >= k, unique and order-independent).
* rounds: the set-by-set restatement of Sec. 1's round rule (``brute.py``).
* IBLT: recovered set == inserted set iff the 2-core of the key hypergraph is
  empty (Sec. 6); per-round recovery == per-round edge removal of the k=2 peel
  on the same hypergraph; XOR/count residue invariants after a failed decode.
* hash convention: the published SplitMix64 vector (finaliser and seed
  stream), the boundaries of the range map (keys with a chosen hash, made by
  inverting mix64), and the frozen known-answer file.
* checksum field: Sec. 6's XOR (insertion and deletion are the same XOR).
"""
import itertools

import numpy as np
import pytest

import oracle
import ppgen
from conftest import read_golden
from oracle import brute


def _rand_hypergraph(rng, n, r, m, distinct=False):
    if distinct:
        return np.array([rng.choice(n, size=r, replace=False) for _ in range(m)],
                        dtype=np.uint32).reshape(m, r)
    return rng.integers(0, n, size=(m, r), dtype=np.uint32)


# ----------------------------------------------------------------------------
# hash convention
# ----------------------------------------------------------------------------
def test_mix64_published_splitmix_vector():
    row = read_golden("splitmix64_published.txt")[0]
    seed, want = int(row[0]), [int(x) for x in row[1:]]
    g = ppgen.SPLITMIX_GAMMA
    got = [oracle.mix64((seed + (i + 1) * g) & ((1 << 64) - 1)) for i in range(5)]
    assert got == want


def test_hash_seeds_are_splitmix_outputs():
    seeds = oracle.hash_seeds(0x13027014, 3)
    assert [int(s) for s in seeds] == [int(x) for x in ppgen.splitmix64_stream(0x13027014, 4)]
    # s_0..s_r are outputs 1..r+1 of SplitMix64 started at the table seed: for
    # the published generator's seed they are its published outputs
    row = read_golden("splitmix64_published.txt")[0]
    assert [int(s) for s in oracle.hash_seeds(int(row[0]), 4)] == [int(x) for x in row[1:6]]


_C1, _C2 = 0xBF58476D1CE4E5B9, 0x94D049BB133111EB
_M64 = (1 << 64) - 1


def _unshift_right(y, s):
    # inverse of z -> z ^ (z >> s) on 64 bits
    z = y
    for _ in range(64 // s + 1):
        z = y ^ (z >> s)
    return z & _M64


def _unmix64(h):
    # inverse of the SplitMix64 finaliser: undo each xorshift and multiply by
    # the inverse of each odd constant mod 2^64
    z = _unshift_right(h, 31)
    z = (z * pow(_C2, -1, 1 << 64)) & _M64
    z = _unshift_right(z, 27)
    z = (z * pow(_C1, -1, 1 << 64)) & _M64
    return _unshift_right(z, 30)


def test_cell_map_boundaries():
    # The cell map splits the 2^64 hash values of sub-table j into size_j
    # intervals of equal width, in order: hash 0 goes to the first cell, 2^64-1
    # to the last, and cell k starts at the first h with h * size >= k * 2^64.
    # Keys with a chosen hash are made by inverting mix64 (a bijection).
    for n, r, seed in [(1000, 3, 5), (4096, 4, 7), (257, 5, 9), ((1 << 26), 3, 0x13027014)]:
        seeds = [int(s) for s in oracle.hash_seeds(seed, r)]
        offs = [int(o) for o in oracle.part_offsets(n, r)]
        for j in range(r):
            size = offs[j + 1] - offs[j]
            probes = [(0, 0), (_M64, size - 1)]
            for k in (1, size // 3, size // 2, size - 1):
                if k <= 0:
                    continue
                first = -(-(k << 64) // size)      # ceil(k 2^64 / size)
                probes += [(first, k), (first - 1, k - 1)]
            for h, want in probes:
                x = _unmix64(h) ^ seeds[j]
                assert oracle.mix64(x ^ seeds[j]) == h
                got = int(oracle.key_cells(n, r, seed, np.array([x], np.uint64))[0][j])
                assert got == offs[j] + want, (n, r, j, h)


def test_part_offsets_headline():
    # 2^26 cells in 3 sub-tables: floor(n/3) + [j < n mod 3]
    off = oracle.part_offsets(1 << 26, 3)
    assert list(np.diff(off)) == [22369622, 22369621, 22369621]
    assert list(np.diff(oracle.part_offsets(10, 4))) == [3, 3, 2, 2]


def test_hash_known_answers():
    rows = read_golden("hash_kat.txt")
    table = None
    for row in rows:
        if row[0] == "table":
            n, r, seed = int(row[1]), int(row[2]), int(row[3])
            bar = row.index("|", 5)
            seeds = [int(x) for x in row[5:bar]]
            offs = [int(x) for x in row[bar + 1:]]
            assert [int(x) for x in oracle.hash_seeds(seed, r)] == seeds
            assert [int(x) for x in oracle.part_offsets(n, r)] == offs
            table = (n, r, seed, offs)
        else:
            n, r, seed, offs = table
            x = int(row[1])
            bar = row.index("|", 3)
            cells = [int(c) for c in row[3:bar]]
            got = oracle.key_cells(n, r, seed, np.array([x], dtype=np.uint64))[0]
            assert [int(c) for c in got] == cells
            for j, c in enumerate(cells):   # one cell per sub-table (App. B)
                assert offs[j] <= c < offs[j + 1]
            assert oracle.checksum(seed, r, x) == int(row[bar + 1])


def test_cell_map_is_multiply_shift():
    # cell_j(x) = off_j + floor(mix64(x ^ s_j) * size_j / 2^64), restated in Python ints
    n, r, seed = 1000, 3, 5
    seeds = [int(s) for s in oracle.hash_seeds(seed, r)]
    offs = [int(o) for o in oracle.part_offsets(n, r)]
    keys = ppgen.distinct_keys(200, 9)
    got = oracle.key_cells(n, r, seed, keys)
    for x, row in zip(keys, got):
        for j in range(r):
            h = ppgen.splitmix64_mix_int(int(x) ^ seeds[j])
            assert int(row[j]) == offs[j] + (h * (offs[j + 1] - offs[j]) >> 64)


# ----------------------------------------------------------------------------
# k-core: brute force, queue peeler, round simulator
# ----------------------------------------------------------------------------
HANDMADE = [
    ("empty graph", 5, 2, np.zeros((0, 3), np.uint32)),
    ("single edge", 3, 2, np.array([[0, 1, 2]], np.uint32)),
    ("two identical edges", 4, 2, np.array([[0, 1, 2], [0, 1, 2]], np.uint32)),
    ("k=1 keeps every edge", 4, 1, np.array([[0, 1, 2], [1, 2, 3]], np.uint32)),
    ("star", 6, 2, np.array([[0, 1], [0, 2], [0, 3], [0, 4], [0, 5]], np.uint32)),
    ("cycle r=2 k=2", 5, 2, np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 0]], np.uint32)),
    ("cycle r=2 k=3", 5, 3, np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 0]], np.uint32)),
    ("K4 r=2 k=3", 4, 3, np.array(list(itertools.combinations(range(4), 2)), np.uint32)),
    ("repeated vertex in an edge", 3, 2, np.array([[0, 0, 1], [1, 2, 2]], np.uint32)),
    ("path of triangles", 7, 2, np.array([[0, 1, 2], [2, 3, 4], [4, 5, 6]], np.uint32)),
]


@pytest.mark.parametrize("name,n,k,edges", HANDMADE, ids=[h[0] for h in HANDMADE])
def test_handmade_cores(name, n, k, edges):
    bv, be = brute.kcore_bruteforce(n, k, edges)
    vc, ec = oracle.kcore_queue(n, k, edges)
    res = oracle.kcore_rounds(n, k, edges)
    assert set(np.nonzero(vc)[0]) == set(bv)
    assert set(np.nonzero(ec)[0]) == set(be)
    assert set(np.nonzero(res["vround"] == 0)[0]) == set(bv)
    assert set(np.nonzero(res["eround"] == 0)[0]) == set(be)
    sv, se, s, m, T = brute.rounds_by_sets(n, k, edges)
    assert list(res["vround"]) == sv and list(res["eround"]) == se
    assert res["s"] == s and res["m"] == m and res["rounds"] == T


def test_handmade_expected_values():
    # two identical triples form a 2-core (Sec. 3's remark on duplicate edges)
    vc, ec = oracle.kcore_queue(4, 2, np.array([[0, 1, 2], [0, 1, 2]], np.uint32))
    assert list(vc) == [1, 1, 1, 0] and list(ec) == [1, 1]
    # a 5-cycle is its own 2-core and has an empty 3-core
    cyc = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 0]], np.uint32)
    assert oracle.kcore_queue(5, 2, cyc)[0].all()
    assert not oracle.kcore_queue(5, 3, cyc)[0].any()
    # path of triangles: leaves go in round 1, the middle edge's outer vertices
    # are then left with degree 1 and go in round 2
    res = oracle.kcore_rounds(7, 2, np.array([[0, 1, 2], [2, 3, 4], [4, 5, 6]], np.uint32))
    assert list(res["vround"]) == [1, 1, 2, 1, 2, 1, 1]
    assert list(res["eround"]) == [1, 1, 1] and res["rounds"] == 2
    assert res["s"] == [2, 0] and res["m"] == [0, 0]


def test_random_tiny_hypergraphs_vs_brute_force():
    rng = np.random.default_rng(1302)
    cases = 0
    for n in range(1, 11):
        for r in (2, 3, 4):
            for k in (1, 2, 3):
                for _ in range(6):
                    m = int(rng.integers(0, 2 * n + 1))
                    edges = _rand_hypergraph(rng, n, r, m)
                    bv, be = brute.kcore_bruteforce(n, k, edges)
                    vc, ec = oracle.kcore_queue(n, k, edges)
                    res = oracle.kcore_rounds(n, k, edges)
                    assert set(np.nonzero(vc)[0]) == set(bv)
                    assert set(np.nonzero(ec)[0]) == set(be)
                    assert set(np.nonzero(res["vround"] == 0)[0]) == set(bv)
                    sv, se, s, mm, T = brute.rounds_by_sets(n, k, edges)
                    assert list(res["vround"]) == sv and list(res["eround"]) == se
                    assert res["s"] == s and res["m"] == mm and res["rounds"] == T
                    cases += 1
    assert cases == 10 * 3 * 3 * 6


def test_exhaustive_two_edge_graphs_r2():
    # every multigraph with 3 edges on 4 vertices, k = 1..3
    pairs = list(itertools.combinations_with_replacement(range(4), 2))
    for es in itertools.combinations_with_replacement(pairs, 3):
        edges = np.array(es, np.uint32)
        for k in (1, 2, 3):
            bv, be = brute.kcore_bruteforce(4, k, edges)
            res = oracle.kcore_rounds(4, k, edges)
            assert set(np.nonzero(res["vround"] == 0)[0]) == set(bv)
            assert set(np.nonzero(res["eround"] == 0)[0]) == set(be)


def test_rounds_medium_vs_sets():
    rng = np.random.default_rng(7)
    for r, k in ((3, 2), (4, 2), (2, 3), (3, 3)):
        n = 300
        m = int(0.9 * n)
        edges = _rand_hypergraph(rng, n, r, m, distinct=True)
        res = oracle.kcore_rounds(n, k, edges)
        sv, se, s, mm, T = brute.rounds_by_sets(n, k, edges)
        assert list(res["vround"]) == sv and list(res["eround"]) == se and res["rounds"] == T
        vc, ec = oracle.kcore_queue(n, k, edges)
        assert (vc == (res["vround"] == 0)).all() and (ec == (res["eround"] == 0)).all()


def test_invalid_vertex_id_rejected():
    with pytest.raises(ValueError):
        oracle.kcore_rounds(3, 2, np.array([[0, 1, 3]], np.uint32))


# ----------------------------------------------------------------------------
# IBLT
# ----------------------------------------------------------------------------
def _iblt(n, r, c, seed, key_seed):
    m = ppgen.edges_from_c(c, n)
    keys = ppgen.distinct_keys(m, key_seed)
    t = oracle.IBLT(n, r, seed)
    t.insert(keys)
    return t, keys


def test_iblt_build_definition():
    # Sec. 6 "Motivation": inserting x XORs x into the key field and checkSum(x)
    # into the checksum field of each of its r cells, and adds 1 to the count.
    n, r, seed = 500, 3, 11
    t, keys = _iblt(n, r, 0.6, seed, 12)
    cells = oracle.key_cells(n, r, seed, keys)
    cnt = np.zeros(n, np.int64)
    kx = np.zeros(n, np.uint64)
    cx = np.zeros(n, np.uint64)
    s_chk = int(oracle.hash_seeds(seed, r)[r])
    for x, row in zip(keys, cells):
        # checkSum(x) is the (published-pinned) mix64 finaliser of x ^ s_chk
        cs = oracle.mix64(int(x) ^ s_chk)
        assert oracle.checksum(seed, r, int(x)) == cs
        for c in row:
            cnt[c] += 1
            kx[c] ^= x
            cx[c] ^= np.uint64(cs)
    assert (t.count == cnt).all() and (t.keyx == kx).all() and (t.chkx == cx).all()
    # deletion undoes insertion; deleting everything empties the table
    t.insert(keys, sign=-1)
    assert not t.count.any() and not t.keyx.any() and not t.chkx.any()


def test_iblt_checksum_field_is_an_xor():
    # Insertion and deletion are the same XORs on both fields (Sec. 6
    # "Motivation"); only the count tells them apart.  A sum would give
    # 2 checkSum(x) after a double insertion and -checkSum(x) after a deletion.
    n, r, seed = 64, 3, 3
    x = np.array([0x0123456789ABCDEF], np.uint64)
    cs = oracle.checksum(seed, r, int(x[0]))
    cells = [int(c) for c in oracle.key_cells(n, r, seed, x)[0]]
    t = oracle.IBLT(n, r, seed)
    t.insert(x)
    assert [int(t.chkx[c]) for c in cells] == [cs] * r
    t.insert(x)      # the same key twice: both XOR fields cancel, count 2
    assert [int(t.chkx[c]) for c in cells] == [0] * r
    assert [int(t.keyx[c]) for c in cells] == [0] * r
    assert [int(t.count[c]) for c in cells] == [2] * r
    u = oracle.IBLT(n, r, seed)
    u.insert(x, sign=-1)     # a deletion of an absent key: same fields, count -1
    assert [int(u.chkx[c]) for c in cells] == [cs] * r
    assert [int(u.keyx[c]) for c in cells] == [int(x[0])] * r
    assert [int(u.count[c]) for c in cells] == [-1] * r
    # the field is the XOR of the checksums whatever the order of insertion
    ks = ppgen.distinct_keys(40, 77)
    a, b = oracle.IBLT(n, r, seed), oracle.IBLT(n, r, seed)
    a.insert(ks)
    b.insert(ks[::-1].copy())
    assert (a.chkx == b.chkx).all()
    want = 0
    for k in ks.tolist():
        if 0 in [int(c) for c in oracle.key_cells(n, r, seed, np.array([k], np.uint64))[0]]:
            want ^= oracle.checksum(seed, r, k)
    assert int(a.chkx[0]) == want


@pytest.mark.parametrize("n,r,c", [(3000, 3, 0.6), (3000, 4, 0.7), (2048, 3, 0.75), (999, 5, 0.6)])
def test_iblt_below_threshold_recovers_inserted_set(n, r, c):
    t, keys = _iblt(n, r, c, 21, 22)
    res = t.decode_rounds()
    got = np.concatenate(res["keys"]) if res["keys"] else np.zeros(0, np.uint64)
    edges = oracle.key_cells(n, r, 21, keys).astype(np.uint32)
    vc, ec = oracle.kcore_queue(n, 2, edges)
    if not ec.any():        # empty 2-core <=> full recovery (Sec. 6)
        assert sorted(got.tolist()) == sorted(keys.tolist())
        assert t.residual_cells() == 0
    assert len(set(got.tolist())) == got.size


@pytest.mark.parametrize("n,r,c,seed", [(4000, 3, 0.7, 1), (4000, 3, 0.9, 2), (3000, 4, 0.85, 3),
                                        (256, 3, 0.7, 4), (600, 2, 0.4, 5)])
def test_iblt_rounds_equal_kcore_rounds(n, r, c, seed):
    # Decoding is the k=2 peel of the key hypergraph (Sec. 6): keys recovered in
    # round t are exactly the edges removed in round t.
    t, keys = _iblt(n, r, c, seed, seed + 100)
    res = t.decode_rounds()
    edges = oracle.key_cells(n, r, seed, keys).astype(np.uint32)
    kc = oracle.kcore_rounds(n, 2, edges)
    by_round = {}
    for x, er in zip(keys.tolist(), kc["eround"].tolist()):
        by_round.setdefault(er, []).append(x)
    T_iblt = max([e for e in by_round if e > 0], default=0)
    assert res["rounds"] == T_iblt
    for i, ks in enumerate(res["keys"], start=1):
        assert sorted(ks.tolist()) == sorted(by_round.get(i, []))
        assert list(ks) == sorted(ks.tolist())
    # cells_alive[t-1] = vertices left after round t of the k = 2 peel
    assert res["cells_alive"] == kc["s"][:res["rounds"]]
    # the residue is the 2-core: non-empty cells == core vertices with edges
    assert t.residual_cells() == len(set(edges[kc["eround"] == 0].ravel().tolist()))


def test_iblt_residue_invariants_above_threshold():
    n, r, seed = 6000, 3, 31
    t, keys = _iblt(n, r, 0.9, seed, 32)
    res = t.decode_rounds()
    got = set(np.concatenate(res["keys"]).tolist())
    left = [x for x in keys.tolist() if x not in got]
    assert left, "c = 0.9 > c*_{2,3} must leave a non-empty core"
    offs = [int(o) for o in oracle.part_offsets(n, r)]
    for j in range(r):                      # each key sits once in every sub-table
        part = slice(offs[j], offs[j + 1])
        assert int(t.count[part].sum()) == len(left)
        x = 0
        for k in left:
            x ^= k
        assert int(np.bitwise_xor.reduce(t.keyx[part])) == x
        cx = 0
        for k in left:
            cx ^= oracle.checksum(seed, r, k)
        assert int(np.bitwise_xor.reduce(t.chkx[part])) == cx
    # no pure cell is left
    for c in range(n):
        assert not (t.count[c] == 1 and int(t.chkx[c]) == oracle.checksum(seed, r, int(t.keyx[c])))


def test_iblt_queue_and_rounds_agree():
    for n, r, c, s in ((5000, 3, 0.8, 41), (5000, 3, 0.85, 42), (4096, 4, 0.78, 43)):
        t1, keys = _iblt(n, r, c, s, s + 1)
        t2 = t1.copy()
        res = t1.decode_rounds()
        q, st = t2.decode_queue()
        assert st == 0
        rounds_set = set(np.concatenate(res["keys"]).tolist()) if res["keys"] else set()
        assert rounds_set == set(q.tolist())
        assert (t1.count == t2.count).all() and (t1.keyx == t2.keyx).all()


def test_iblt_duplicate_cells_make_a_core():
    # two keys with identical cell triples can never be peeled (Sec. 3 remark)
    n, r, seed = 9, 3, 77
    rng = np.random.default_rng(0)
    cand = ppgen.distinct_keys(200000, 5)
    cells = oracle.key_cells(n, r, seed, cand)
    seen = {}
    pair = None
    for x, row in zip(cand.tolist(), map(tuple, cells.tolist())):
        if row in seen:
            pair = (seen[row], x)
            break
        seen[row] = x
    assert pair is not None
    t = oracle.IBLT(n, r, seed)
    t.insert(np.array(pair, np.uint64))
    res = t.decode_rounds()
    assert res["rounds"] == 0 and t.residual_cells() == 3
    del rng


def test_iblt_empty_table():
    t = oracle.IBLT(64, 3, 1)
    res = t.decode_rounds()
    assert res["rounds"] == 0 and res["keys"] == []


def test_iblt_below_threshold_recovered_inserted_set_wrapper():
    for n, r, c in [(3000, 3, 0.6), (3000, 4, 0.7), (999, 5, 0.6)]:
        test_iblt_below_threshold_recovers_inserted_set(n, r, c)


def test_iblt_checksum_rejects_impure_count_one():
    # With deletions a cell can reach count 1 while holding a mixture of keys
    # (+a +b -c).  Only pure cells may release a key (Sec. 6), and the checksum
    # field is what tells them apart: every recovered key must be a real key.
    n, r, seed = 60, 3, 5
    ins = ppgen.distinct_keys(45, 101)
    dele = ppgen.distinct_keys(30, 202)
    t = oracle.IBLT(n, r, seed)
    t.insert(ins)
    t.insert(dele, sign=-1)
    mixed = 0
    for c in range(n):
        if t.count[c] == 1 and int(t.chkx[c]) != oracle.checksum(seed, r, int(t.keyx[c])):
            mixed += 1
    assert mixed > 0
    res = t.decode_rounds()
    got = np.concatenate(res["keys"]).tolist() if res["keys"] else []
    assert set(got) <= set(ins.tolist())
