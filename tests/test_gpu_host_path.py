"""GPU: build + decode from host buffers (pp_iblt_submit_host /
pp_iblt_finish_host / pp_iblt_build_decode_host) against the CPU oracle:
each round's key set, the rounds, the per-round survivors, the residue."""
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


def _pinned(n):
    return torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)


def _check(res, out, n, r, seed, keys):
    ot = oracle.IBLT(n, r, seed)
    ot.insert(keys)
    ores = ot.decode_rounds()
    assert res.rounds == ores["rounds"]
    assert res.recovered_per_round == [k.size for k in ores["keys"]]
    assert res.alive_cells_per_round == ores["cells_alive"]
    assert res.residual_cells == ot.residual_cells()
    ends = np.cumsum([0] + res.recovered_per_round)
    for t, k in enumerate(ores["keys"]):
        assert (np.sort(out[ends[t]:ends[t + 1]]) == k).all(), t


@pytest.mark.parametrize("n,r,c,pinned", [(5000, 3, 0.7, True), (70001, 4, 0.85, False),
                                          ((1 << 21) + 9, 3, 0.75, True), ((1 << 21) + 9, 3, 0.8, False)])
def test_build_decode_host(pp, n, r, c, pinned):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), n + 3)
    if pinned:
        hk = _pinned(keys.size)
        hk[:] = keys
        out = _pinned(keys.size)
    else:
        hk, out = keys.copy(), np.zeros(keys.size, np.uint64)
    t = pp.IBLT(n, r, 11)
    res = t.build_decode_host(hk, out)
    _check(res, out, n, r, 11, keys)
    t.close()


def test_jobs_in_flight(pp):
    n, r = (1 << 21) + 33, 3
    t = pp.IBLT(n, r, 5)
    specs = [(0.7, 1), (0.8, 2), (0.5, 3), (0.9, 4), (0.6, 5), (0.75, 6)]
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(c, n), s) for c, s in specs]
    hk = [_pinned(k.size) for k in keys]
    outs = [_pinned(k.size) for k in keys]
    for h, k in zip(hk, keys):
        h[:] = k
    tickets = [t.submit_host(hk[i], outs[i]) for i in range(3)]
    with pytest.raises(pp.PPError) as ei:
        t.submit_host(hk[3], outs[3])      # a fourth job while three are in flight
    assert ei.value.name == "PP_ERR_INVALID_ARG"
    results = {}
    for i in range(len(specs)):
        results[i] = t.finish_host(tickets[i])
        if i + 3 < len(specs):
            tickets.append(t.submit_host(hk[i + 3], outs[i + 3]))
    for i, k in enumerate(keys):
        _check(results[i], outs[i], n, r, 5, k)
    t.close()


def test_slab_overflow_job_is_redone(pp):
    """Keys whose first cell all falls in the first 2^21-cell slab overfill that
    slab's list in the binned build; the job comes back right all the same."""
    n, r, seed = 1 << 23, 3, 7
    cand = ppgen.distinct_keys(3_000_000, 8)
    first = oracle.key_cells(n, r, seed, cand)[:, 0]
    keys = cand[first < (1 << 21)]
    hk = _pinned(keys.size)
    hk[:] = keys
    out = _pinned(keys.size)
    t = pp.IBLT(n, r, seed)
    ticket = t.submit_host(hk, out)
    other = ppgen.distinct_keys(ppgen.edges_from_c(0.5, n), 9)   # a normal job behind it
    hk2 = _pinned(other.size)
    hk2[:] = other
    out2 = _pinned(other.size)
    t2 = t.submit_host(hk2, out2)
    _check(t.finish_host(ticket), out, n, r, seed, keys)
    _check(t.finish_host(t2), out2, n, r, seed, other)
    t.close()


def test_host_path_capacity(pp):
    keys = ppgen.distinct_keys(1000, 3)
    t = pp.IBLT(3000, 3, 1)
    with pytest.raises(pp.PPError) as ei:
        t.submit_host(keys, np.zeros(999, np.uint64))
    assert ei.value.name == "PP_ERR_CAPACITY"
    with pytest.raises(pp.PPError):
        t.finish_host(12345)              # no such job
    t.close()
