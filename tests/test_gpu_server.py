"""GPU tests of the continuous-batching decode service.

Each request's result must be exactly the oracle's decode of that request
alone (rounds, keys recovered, residue) even though many requests share the
device and join each other's rounds mid-flight.
"""
import time

import numpy as np
import pytest

import oracle
import ppgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def srv_mod(ppeel_lib):
    import paper_1302_7014_b300 as pp
    import paper_1302_7014_b300.server as server
    return pp, server


def _oracle(spec, keys):
    n, r, c, tseed, kseed = spec
    ot = oracle.IBLT(n, r, tseed)
    ot.insert(keys)
    res = ot.decode_rounds()
    got = np.concatenate(res["keys"]) if res["keys"] else np.zeros(0, np.uint64)
    return res["rounds"], got, ot.residual_cells()


def _specs(count, seed, lo=8, hi=16, rs=(3,), c_lo=0.5, c_hi=0.95):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(2 ** rng.uniform(lo, hi))
        r = int(rng.choice(rs))
        out.append((max(n, r), r, float(rng.uniform(c_lo, c_hi)), int(rng.integers(1, 2**62)),
                    int(rng.integers(1, 2**62))))
    return out


def _check(res, spec, keys):
    rounds, want, residual = _oracle(spec, keys)
    assert res["status"] == 0
    assert res["rounds"] == rounds
    assert res["recovered"] == want.size
    assert res["residual_cells"] == residual
    assert res["items_before"] == keys.size
    if "keys" in res:
        assert (np.sort(res["keys"]) == np.sort(want)).all()
    assert res["done_s"] >= res["admit_s"] >= res["arrival_s"] > 0


@pytest.mark.parametrize("r_cfg", [0, 3])
def test_results_equal_alone_in_the_mix(srv_mod, r_cfg):
    pp, server = srv_mod
    specs = _specs(48, 11 + r_cfg, rs=(3,) if r_cfg else (2, 3, 4, 5))
    s = server.Server(arena_cells=1 << 22, arena_keys=1 << 22, max_slots=256, r=r_cfg)
    tickets = []
    for i, sp in enumerate(specs):
        n, r, c, tseed, kseed = sp
        m = ppgen.edges_from_c(c, n)
        if i % 2:   # host keys
            keys = ppgen.distinct_keys(m, kseed)
            tickets.append((s.submit(n, r, tseed, m, keys=keys, want_keys=True), sp, keys))
        else:       # synthetic keys: SplitMix64 stream from key_seed, generated on the device
            tickets.append((s.submit(n, r, tseed, m, key_seed=kseed, want_keys=True), sp,
                            ppgen.distinct_keys(m, kseed)))
    for t, sp, keys in tickets:
        _check(s.wait(t, 60.0), sp, keys)
    st = s.stats()
    assert st["completed"] == len(specs) and st["pending"] == 0 and st["active"] == 0
    # the same requests one at a time on the now idle server give the same results
    for t, sp, keys in tickets[:6]:
        n, r, c, tseed, kseed = sp
        res = s.wait(s.submit(n, r, tseed, keys.size, keys=keys, want_keys=True), 60.0)
        _check(res, sp, keys)
    s.stop()


def test_admission_by_free_memory(srv_mod):
    pp, server = srv_mod
    # the arena holds only a few tables at once: requests queue and cycle through it
    specs = _specs(40, 5, lo=10, hi=12.5)
    s = server.Server(arena_cells=1 << 13, arena_keys=1 << 13, max_slots=8, r=3)
    tickets = [(s.submit(sp[0], sp[1], sp[3], ppgen.edges_from_c(sp[2], sp[0]), key_seed=sp[4]), sp)
               for sp in specs]
    for t, sp in tickets:
        keys = ppgen.distinct_keys(ppgen.edges_from_c(sp[2], sp[0]), sp[4])
        _check(s.wait(t, 60.0), sp, keys)
    st = s.stats()
    assert st["admitted"] == 40 and st["iterations"] > 40
    # time accounting: every iteration waits on the GPU for part of its time
    assert 0 < st["gpu_wait_us"] <= st["iteration_us"]
    s.stop()


def test_rejections_and_timeout(srv_mod):
    pp, server = srv_mod
    s = server.Server(arena_cells=1 << 12, arena_keys=1 << 12, max_slots=4, r=3)
    with pytest.raises(pp.PPError) as ei:
        s.submit(1 << 13, 3, 1, 100)                 # larger than the cell arena
    assert ei.value.name == "PP_ERR_CAPACITY"
    with pytest.raises(pp.PPError) as ei:
        s.submit(1000, 4, 1, 100)                    # this server only serves r = 3
    assert ei.value.name == "PP_ERR_INVALID_ARG"
    t = s.submit(4000, 3, 7, 3000, key_seed=8)
    with pytest.raises(pp.PPError) as ei:
        s.wait(t, 1e-6)                              # cannot be done a microsecond later
    assert ei.value.name == "PP_ERR_TIMEOUT"
    res = s.wait(t, 60.0)
    assert res["recovered"] <= 3000
    with pytest.raises(pp.PPError) as ei:
        s.wait(t, 1.0)                               # the ticket was released
    assert ei.value.name == "PP_ERR_NOT_FOUND"
    s.stop()


def test_stop_without_drain_returns(srv_mod):
    pp, server = srv_mod
    s = server.Server(arena_cells=1 << 16, arena_keys=1 << 16, max_slots=16, r=3)
    for i in range(200):
        s.submit(4000, 3, i, 3000, key_seed=i)
    t0 = time.time()
    s.stop(drain=False)
    assert time.time() - t0 < 30


def test_poisson_arrivals_small(srv_mod):
    pp, server = srv_mod
    reqs = ppgen.serving_requests(300, rate_per_s=3000.0, lo_log2=10, hi_log2=16)
    s = server.Server(arena_cells=1 << 22, arena_keys=1 << 22, max_slots=512, r=3)
    t0 = server.server_now()
    tickets = []
    for at, spec in reqs:
        while server.server_now() - t0 < at:
            pass
        tickets.append((s.submit(spec.n_cells, spec.r, spec.table_seed, spec.m, key_seed=spec.key_seed,
                                 arrival_s=t0 + at), spec))
    lat = []
    for t, spec in tickets:
        res = s.wait(t, 60.0)
        lat.append(res["done_s"] - res["arrival_s"])
    # spot-check results against the oracle
    s2 = server.Server(arena_cells=1 << 22, arena_keys=1 << 22, max_slots=64, r=3)
    for at, spec in reqs[::37]:
        keys = spec.keys()
        res = s2.wait(s2.submit(spec.n_cells, 3, spec.table_seed, spec.m, keys=keys, want_keys=True), 60.0)
        _check(res, (spec.n_cells, 3, spec.c, spec.table_seed, spec.key_seed), keys)
    s2.stop()
    s.stop()
    assert len(lat) == 300 and max(lat) < 30.0
