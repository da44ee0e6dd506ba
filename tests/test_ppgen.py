"""The shared input generators: scalar definitions vs the fast C streams."""
import numpy as np

import ppgen
from conftest import read_golden


def test_splitmix64_published_vector():
    # tests/golden/splitmix64_published.txt: reference outputs for seed 1234567
    row = read_golden("splitmix64_published.txt")[0]
    seed, want = int(row[0]), [int(x) for x in row[1:]]
    assert [int(x) for x in ppgen.splitmix64_stream(seed, 5)] == want
    assert [ppgen.splitmix64_mix_int(seed + (i + 1) * ppgen.SPLITMIX_GAMMA) for i in range(5)] == want


def test_splitmix64_offset_stream():
    a = ppgen.splitmix64_stream(99, 1000)
    b = ppgen.splitmix64_stream(99, 10, start=990)
    assert (a[990:] == b).all()


def test_xorshift64star_matches_scalar():
    for seed in (0, 1, 7, 2**63 + 5):
        g = ppgen.XorShift64Star(seed)
        ref = np.array([g.next() for _ in range(3000)], dtype=np.uint64)
        assert (ppgen.xorshift64star_stream(seed, 3000) == ref).all()
        assert (ppgen.xorshift64star_stream(seed, 17) == ref[:17]).all()


def test_keys_distinct():
    k = ppgen.distinct_keys(1 << 20, 2)
    assert np.unique(k).size == k.size


def test_partitioned_edges_layout():
    n, r, m = 1 << 14, 3, ppgen.edges_from_c(0.70, 1 << 14)
    assert m == 11468
    e = ppgen.partitioned_edges(n, r, m, 1)
    offs = ppgen.part_offsets(n, r)
    assert ppgen.part_sizes(n, r) == [5462, 5461, 5461]
    draws = ppgen.xorshift64star_stream(1, m * r).reshape(m, r)
    for j in range(r):
        assert (e[:, j] >= offs[j]).all() and (e[:, j] < offs[j + 1]).all()
        want = ppgen.mulhi_u64_u32(draws[:, j], offs[j + 1] - offs[j]) + np.uint64(offs[j])
        assert (e[:, j] == want).all()


def test_distinct_uniform_edges():
    e = ppgen.distinct_uniform_edges(50, 4, 2000, 3)
    s = np.sort(e, axis=1)
    assert not (s[:, 1:] == s[:, :-1]).any()
    assert e.max() < 50


def test_recipe_sizes():
    # m = floor(c n) for the density sweep at n = 2^25
    n = ppgen.DENSITY_SWEEP["n"]
    ms = [ppgen.edges_from_c(c, n) for c in ppgen.DENSITY_SWEEP["cs"]]
    assert ms == [23488102, 25501368, 26172456, 26843545, 28521267]
    assert ppgen.edges_from_c(0.75, 1 << 26) == 50331648


def test_batch_recipe():
    tabs = ppgen.batch_tables(4096)
    assert len(tabs) == 4096
    assert all(256 <= t.n_cells < (1 << 20) for t in tabs)
    assert {t.r for t in tabs} == {3, 4}
    for t in tabs:
        assert 0.5 <= t.c <= 0.9 * ppgen.CSTAR_PRINTED[t.r]
        assert t.m == int(t.c * t.n_cells)
    # log-uniform sizes: about half the tables below 2^14 cells
    frac = np.mean([t.n_cells < (1 << 14) for t in tabs])
    assert 0.45 < frac < 0.55


def test_serving_recipe():
    reqs = ppgen.serving_requests(20000, rate_per_s=20000.0)
    times = np.array([t for t, _ in reqs])
    gaps = np.diff(times)
    assert abs(gaps.mean() * 20000.0 - 1.0) < 0.05
    assert all(1024 <= s.n_cells < (1 << 22) and s.r == 3 and 0.6 <= s.c <= 0.8 for _, s in reqs)


def test_trials_union_is_a_disjoint_union():
    import oracle
    n, r, m, T = 300, 4, 210, 7
    for kind in ("distinct", "partitioned"):
        e, uoff, to_trials = ppgen.trials_union(n, r, m, T, 5, kind)
        assert e.shape == (m * T, r)
        if kind == "partitioned":
            assert uoff == [T * o for o in ppgen.part_offsets(n, r)[:r]] + [T * n]
            whole = oracle.kcore_subrounds(n * T, 2, e, uoff)
        else:
            assert uoff is None
            whole = oracle.kcore_rounds(n * T, 2, e)
        per = to_trials(whole["vround"])
        # each trial, peeled alone, removes the same vertices in the same
        # (sub-)rounds as inside the union
        for i in range(T):
            rows = e[i * m:(i + 1) * m].astype(np.int64)
            if kind == "partitioned":
                offs, sizes = ppgen.part_offsets(n, r), ppgen.part_sizes(n, r)
                local = np.stack([rows[:, j] - T * offs[j] - i * sizes[j] + offs[j] for j in range(r)], axis=1)
                alone = oracle.kcore_subrounds(n, 2, local.astype(np.uint32), offs[:r] + [n])
            else:
                local = rows - i * n
                alone = oracle.kcore_rounds(n, 2, local.astype(np.uint32))
            assert (local >= 0).all() and (local < n).all()
            assert (per[i] == alone["vround"]).all(), (kind, i)
