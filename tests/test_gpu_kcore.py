"""GPU parity: round-synchronous k-core peeling against the CPU oracle.

Exact comparison of each vertex's and edge's removal round, the number of
rounds and the per-round survivor counts s_t and m_t.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import ppgen
from conftest import GOLDEN
import test_oracle_pins as pins

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pp(ppeel_lib):
    import paper_1302_7014_b300 as pp
    return pp


def gpu_peel(pp, n, r, k, edges, opts=None):
    m = edges.shape[0]
    d_edges = torch.from_numpy(np.ascontiguousarray(edges, dtype=np.uint32).view(np.int32)).cuda()
    if m == 0:
        d_edges = torch.zeros((0, r), dtype=torch.int32, device="cuda")
    vr = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    er = torch.full((max(m, 1),), -7, dtype=torch.int32, device="cuda")
    res = pp.peel_kcore(n, r, k, d_edges, vr[:n] if n else None, er[:m] if m else None, opts)
    return res, vr[:n].cpu().numpy(), er[:m].cpu().numpy()


def check(pp, n, k, edges, opts=None):
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    r = edges.shape[1]
    res, vr, er = gpu_peel(pp, n, r, k, edges, opts)
    o = oracle.kcore_rounds(n, k, edges)
    assert res.rounds == o["rounds"]
    assert (vr == o["vround"]).all()
    assert (er == o["eround"]).all()
    assert res.vertices_left == o["s"] and res.edges_left == o["m"]
    assert res.core_vertices == int((o["vround"] == 0).sum())
    assert res.core_edges == int((o["eround"] == 0).sum())
    return res


@pytest.mark.parametrize("name,n,k,edges", pins.HANDMADE, ids=[h[0] for h in pins.HANDMADE])
def test_handmade(pp, name, n, k, edges):
    if edges.shape[1] < 2:
        pytest.skip("r >= 2")
    check(pp, n, k, edges)


def test_random_small(pp):
    rng = np.random.default_rng(2024)
    for trial in range(60):
        n = int(rng.integers(1, 3000))
        r = int(rng.choice([2, 3, 4, 6]))
        k = int(rng.choice([1, 2, 3, 4]))
        c = float(rng.uniform(0.2, 1.6))
        m = int(c * n)
        edges = ppgen.uniform_edges(n, r, m, 900 + trial)   # repeats inside an edge allowed
        check(pp, n, k, edges)


@pytest.mark.parametrize("n,r,k,c", [(5000, 3, 2, 0.8), (65537, 4, 2, 0.76), (40000, 2, 3, 1.6),
                                     (30011, 3, 3, 1.5), (100000, 4, 2, 0.9), (2 ** 17 + 3, 5, 2, 0.6)])
def test_partitioned(pp, n, r, k, c):
    edges = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(c, n), n + r)
    check(pp, n, k, edges)


def test_host_loop_matches(pp):
    edges = ppgen.partitioned_edges(70000, 4, ppgen.edges_from_c(0.8, 70000), 5)
    check(pp, 70000, 2, edges, opts=pp.options(host_loop=1))
    check(pp, 70000, 2, edges, opts=pp.options(ctas_per_sm=1))


def _hub_edges(n, r, hub, hub_deg, seed):
    """hub_deg edges through vertex `hub` plus filler edges; no other edge
    touches vertices 0 and 1, so deg(hub) == hub_deg exactly."""
    rng = np.random.default_rng(seed)
    e = rng.integers(2, n, size=(hub_deg, r), dtype=np.uint64).astype(np.uint32)
    e[:, 0] = hub
    filler = (ppgen.uniform_edges(n - 2, r, 20000, seed).astype(np.uint64) + 2).astype(np.uint32)
    return np.concatenate([e, filler])


@pytest.mark.parametrize("hub", [0, 1], ids=["low-half", "high-half"])
@pytest.mark.parametrize("hub_deg", [65535, 65536, 70001])
def test_high_degree_vertex(pp, hub_deg, hub):
    """Degrees are counted in the 16-bit halves of 32-bit words; a degree of
    65536 or more carries out of its half and the call counts again in 32
    bits.  Both sides of that boundary, for a vertex in either half."""
    n, r = 50000, 3
    edges = _hub_edges(n, r, hub, hub_deg, hub_deg + hub)
    assert int((edges == hub).sum()) == hub_deg
    for k in (2, 3):
        check(pp, n, k, edges)


MODES = [0, 1, 2]  # auto (edge-centric, then incidence lists), incidence lists only, edge-centric only


@pytest.mark.parametrize("mode", MODES, ids=["auto", "lists", "edges"])
def test_round_modes_random(pp, mode):
    """Every way of running the full rounds gives the oracle's rounds exactly."""
    rng = np.random.default_rng(77 + mode)
    for trial in range(30):
        n = int(rng.integers(2, 5000))
        r = int(rng.choice([2, 3, 4]))
        k = int(rng.choice([1, 2, 3]))
        c = float(rng.uniform(0.2, 1.8))
        edges = ppgen.uniform_edges(n, r, int(c * n), 3100 + trial)
        check(pp, n, k, edges, opts=pp.options(kcore_mode=mode))


@pytest.mark.parametrize("mode", MODES, ids=["auto", "lists", "edges"])
@pytest.mark.parametrize("c", [0.70, 0.76, 0.78, 0.85])
def test_round_modes_density_sweep(pp, mode, c):
    """The density sweep's recipe at 2^20 vertices: below the threshold the
    core is empty after many rounds, above it most edges stay; the automatic
    mode hands over to incidence lists part way (with or without removed
    entries still in the edge list)."""
    cfg = ppgen.DENSITY_SWEEP
    n, r, k = 1 << 20, cfg["r"], cfg["k"]
    edges = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(c, n), cfg["seed"])
    check(pp, n, k, edges, opts=pp.options(kcore_mode=mode))
    if mode == 0:
        check(pp, n, k, edges, opts=pp.options(kcore_mode=mode, host_loop=1))


def check_modes(pp, n, k, edges, modes=MODES, host_loop=True):
    """check() for every mode against one oracle run."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    r = edges.shape[1]
    o = oracle.kcore_rounds(n, k, edges)
    runs = [pp.options(kcore_mode=md) for md in modes]
    if host_loop:
        runs.append(pp.options(kcore_mode=0, host_loop=1))
    for opts in runs:
        res, vr, er = gpu_peel(pp, n, r, k, edges, opts)
        assert res.rounds == o["rounds"]
        assert (vr == o["vround"]).all()
        assert (er == o["eround"]).all()
        assert res.vertices_left == o["s"] and res.edges_left == o["m"]


@pytest.mark.parametrize("dense_c,seed", [(0.85, 1), (0.9, 2), (1.0, 3), (1.3, 4)])
def test_round_modes_mixed_density(pp, dense_c, seed):
    """A sparse part (most vertices go in round 1, so the automatic mode starts
    edge-centric; over 2^20 edges in all) joined to a dense part that leaves a
    slowly peeling core (so it hands over to incidence lists part way, with the
    edge list compacted or holding removed entries, depending on the rounds
    before)."""
    n1, n2, r = 2_000_000, 700_000, 3
    sparse = ppgen.uniform_edges(n1, r, int(0.3 * n1), 40 + seed)
    dense = (ppgen.uniform_edges(n2, r, int(dense_c * n2), 50 + seed).astype(np.uint64) + n1).astype(np.uint32)
    edges = np.concatenate([sparse, dense])
    edges = edges[np.random.default_rng(seed).permutation(edges.shape[0])]
    assert edges.shape[0] >= 1 << 20
    check_modes(pp, n1 + n2, 2, edges)


def test_round_modes_small_first_frontier(pp):
    """A dense graph whose F_1 is tiny: the automatic mode hands over before
    round 1, on the caller's own edge array."""
    n, r = 20000, 3
    edges = ppgen.partitioned_edges(n, r, int(1.5 * n), 11)
    for mode in MODES:
        check(pp, n, 2, edges, opts=pp.options(kcore_mode=mode))


def test_misaligned_edge_array(pp):
    """Rows not 16-byte aligned (an offset view): the generic round kernels run."""
    n, r = 30000, 4
    edges = ppgen.partitioned_edges(n, r, int(0.7 * n), 13)
    m = edges.shape[0]
    buf = torch.zeros(m * r + 1, dtype=torch.int32, device="cuda")
    buf[1:] = torch.from_numpy(np.ascontiguousarray(edges, dtype=np.uint32).view(np.int32).reshape(-1)).cuda()
    d_edges = buf[1:].view(m, r)
    assert d_edges.data_ptr() % 16 != 0
    o = oracle.kcore_rounds(n, 2, edges)
    for mode in MODES:
        vr = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        er = torch.full((m,), -7, dtype=torch.int32, device="cuda")
        res = pp.peel_kcore(n, r, 2, d_edges, vr, er, pp.options(kcore_mode=mode))
        assert res.rounds == o["rounds"]
        assert (vr.cpu().numpy() == o["vround"]).all() and (er.cpu().numpy() == o["eround"]).all()


def test_plain_peel_config(pp):
    cfg = ppgen.PLAIN_PEEL
    n, r, k = cfg["n"], cfg["r"], cfg["k"]
    edges = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(cfg["c"], n), cfg["seed"])
    res = check(pp, n, k, edges)
    assert res.core_vertices == 0 and 8 <= res.rounds <= 20


def test_no_edges(pp):
    res = check(pp, 5, 2, np.zeros((0, 3), np.uint32))
    assert res.rounds == 1 and res.vertices_left == [0]


def test_invalid_vertex_id(pp):
    edges = np.array([[0, 1, 2], [0, 5, 1]], np.uint32)
    with pytest.raises(pp.PPError) as ei:
        gpu_peel(pp, 5, 3, 2, edges)
    assert ei.value.name == "PP_ERR_INVALID_ARG"


def test_round_limit(pp):
    edges = ppgen.partitioned_edges(20000, 3, 14000, 3)
    with pytest.raises(pp.PPError) as ei:
        gpu_peel(pp, 20000, 3, 2, edges, pp.options(max_rounds=2))
    assert ei.value.name == "PP_ERR_ROUND_LIMIT"


@pytest.mark.parametrize("n,r,m,k", [(16384, 4, 65536, 2), (16385, 3, 11000, 2), (16384, 3, 65537, 3),
                                     (1, 2, 3, 1), (300, 8, 700, 2), (4096, 5, 3000, 4)])
def test_small_graph_limits(pp, n, r, m, k):
    # graphs of at most 2^14 vertices and 2^16 edges peel in one block; the
    # cases at and just past both limits take the two paths
    edges = ppgen.uniform_edges(n, r, m, 77 + n + m)
    check(pp, n, k, edges)


@pytest.mark.parametrize("max_rounds", [1, 2, 3])
def test_small_graph_round_limit_matches_lists(pp, max_rounds):
    # the same partial peel from the one-block path (automatic mode), the
    # incidence lists and the edge-centric rounds: rounds 1..max_rounds as the
    # oracle has them, the vertices round max_rounds + 1 would remove marked
    # with that round, everything else 0; the same error from each
    n, r = 12000, 3
    edges = ppgen.partitioned_edges(n, r, 8400, 5)
    d_edges = torch.from_numpy(edges.view(np.int32)).cuda()
    o = oracle.kcore_rounds(n, 2, edges)
    vr_o = np.where(o["vround"] <= max_rounds + 1, o["vround"], 0)
    er_o = np.where(o["eround"] <= max_rounds, o["eround"], 0)
    for mode in (0, 1, 2):
        vr = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        er = torch.full((edges.shape[0],), -7, dtype=torch.int32, device="cuda")
        with pytest.raises(pp.PPError) as ei:
            pp.peel_kcore(n, r, 2, d_edges, vr, er, pp.options(max_rounds=max_rounds, kcore_mode=mode))
        assert ei.value.name == "PP_ERR_ROUND_LIMIT"
        assert (vr.cpu().numpy() == vr_o).all(), mode
        assert (er.cpu().numpy() == er_o).all(), mode


def test_small_graph_without_outputs(pp):
    cfg = ppgen.PLAIN_PEEL
    n, r, k = cfg["n"], cfg["r"], cfg["k"]
    edges = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(cfg["c"], n), cfg["seed"])
    d_edges = torch.from_numpy(edges.view(np.int32)).cuda()
    res = pp.peel_kcore(n, r, k, d_edges)
    o = oracle.kcore_rounds(n, k, edges)
    assert res.rounds == o["rounds"] and res.vertices_left == o["s"] and res.edges_left == o["m"]


def test_small_graph_from_several_threads(pp):
    # the one-block path keeps its result buffer per calling thread: calls from
    # threads of their own (each on its own stream) give the oracle's result,
    # and the threads exit (freeing their buffers) cleanly
    import threading
    cases = [(3000 + 500 * i, 3 + (i % 2), 2, 0.6 + 0.05 * i) for i in range(4)]
    want, got = {}, {}
    for i, (n, r, k, c) in enumerate(cases):
        edges = ppgen.uniform_edges(n, r, int(c * n), 300 + i)
        want[i] = (edges, oracle.kcore_rounds(n, k, edges))

    def work(i):
        n, r, k, _ = cases[i]
        edges = want[i][0]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            d = torch.from_numpy(edges.view(np.int32)).cuda()
            vr = torch.empty(n, dtype=torch.int32, device="cuda")
        s.synchronize()
        for _ in range(20):
            res = pp.peel_kcore(n, r, k, d, vr, None, stream=s)
        got[i] = (res, vr.cpu().numpy())

    ts = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for i in range(len(cases)):
        res, vr = got[i]
        o = want[i][1]
        assert res.rounds == o["rounds"] and res.vertices_left == o["s"] and (vr == o["vround"]).all()


def test_iblt_decode_is_the_k2_peel(pp):
    # Sec. 6: recovery is peeling at k = 2 on the key hypergraph; both GPU paths agree
    n, r, seed = 120000, 3, 88
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.8, n), 89)
    edges = oracle.key_cells(n, r, seed, keys).astype(np.uint32)
    kres, vr, er = gpu_peel(pp, n, r, 2, edges)
    t = pp.IBLT(n, r, seed)
    t.insert(torch.from_numpy(keys.view(np.int64)).cuda())
    out = torch.zeros(keys.size, dtype=torch.int64, device="cuda")
    ires = t.decode(out)
    removed = np.bincount(er[er > 0], minlength=kres.rounds + 1)[1:]
    assert ires.rounds == max([t_ for t_ in range(1, kres.rounds + 1) if removed[t_ - 1]], default=0)
    assert ires.recovered_per_round == [int(x) for x in removed[: ires.rounds]]
    assert ires.alive_cells_per_round == kres.vertices_left[: ires.rounds]


@pytest.mark.parametrize("idx", range(5))
def test_density_sweep_full_size(pp, idx):
    gold = json.load(open(os.path.join(GOLDEN, "full_size.json")))["density_sweep"][idx]
    n, r, k = gold["n"], gold["r"], gold["k"]
    edges = ppgen.partitioned_edges(n, r, gold["m"], gold["seed"])
    res, vr, er = gpu_peel(pp, n, r, k, edges)
    assert res.rounds == gold["rounds"]
    assert res.vertices_left == gold["s"] and res.edges_left == gold["m_t"]
    assert res.core_vertices == gold["core_vertices"] and res.core_edges == gold["core_edges"]
    assert hashlib.sha256(vr.astype("<i4").tobytes()).hexdigest() == gold["vround_sha256"]
    assert hashlib.sha256(er.astype("<i4").tobytes()).hexdigest() == gold["eround_sha256"]
