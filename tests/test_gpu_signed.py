"""GPU parity: signed IBLT recovery of a set difference against the oracle.

Exact comparisons: each round's (key, sign) pairs, the number of rounds, the
residue left in the table bit for bit and the residue count.
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


def _dev(keys):
    return torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()


def _sets(n_a, n_b, n_common, seed):
    keys = ppgen.distinct_keys(n_a + n_b + n_common, seed)
    common = keys[:n_common]
    return np.concatenate([common, keys[n_common:n_common + n_a]]), np.concatenate([common, keys[n_common + n_a:]])


def run_signed(pp, n, r, A, B, seed, opts=None, with_signs=True):
    gt = pp.IBLT(n, r, seed, opts)
    ot = oracle.IBLT(n, r, seed)
    if len(A):
        gt.insert(_dev(A))
        ot.insert(A)
    if len(B):
        gt.delete(_dev(B))
        ot.insert(B, sign=-1)
    cap = max(1, len(A) + len(B))
    out = torch.zeros(cap, dtype=torch.int64, device="cuda")
    sg = torch.zeros(cap, dtype=torch.int8, device="cuda") if with_signs else None
    res = gt.decode_signed(out, sg, round_cap=1 << 14)
    ores = ot.decode_signed()
    assert res.rounds == ores["rounds"]
    keys = out[: res.recovered].cpu().numpy().view(np.uint64)
    signs = sg[: res.recovered].cpu().numpy() if with_signs else None
    ends = np.cumsum([0] + list(res.recovered_per_round))
    assert ends[-1] == res.recovered
    for t, (wk, ws) in enumerate(zip(ores["keys"], ores["signs"])):
        k = keys[ends[t]:ends[t + 1]]
        o = np.argsort(k)
        assert np.array_equal(k[o], wk), t + 1
        if with_signs:
            assert np.array_equal(signs[ends[t]:ends[t + 1]][o], ws), t + 1
    cells = gt.cells()
    assert (cells["count"].astype(np.int64) == ot.count).all()
    assert (cells["key_xor"] == ot.keyx).all() and (cells["chk_xor"] == ot.chkx).all()
    assert res.residual_cells == ot.residual_cells()
    gt.close()
    return res


@pytest.mark.parametrize("n,r,fa,fb,common,seed", [
    (1000, 3, 0.40, 0.30, 500, 1),
    (3 * 1024 + 17, 3, 0.50, 0.25, 4000, 2),
    (50021, 3, 0.45, 0.35, 20000, 3),    # close to the threshold
    (65536, 4, 0.40, 0.30, 30000, 4),
    (40000, 3, 0.60, 0.40, 10000, 5),    # above c*_{2,3}: a residue stays
    (30011, 5, 0.30, 0.30, 5000, 6),     # generic kernel
    (20000, 2, 0.20, 0.20, 5000, 7),
])
@pytest.mark.parametrize("binned", [0, 1], ids=["direct", "binned"])
def test_set_difference(pp, n, r, fa, fb, common, seed, binned):
    """binned=1 forces the binned rounds (claim records carry the sign) on
    tables that would otherwise apply their updates directly."""
    A, B = _sets(int(fa * n), int(fb * n), common, 10 + seed)
    run_signed(pp, n, r, A, B, seed, opts=pp.options(binned=binned))


def test_insert_only_matches_unsigned(pp):
    n, r = 50000, 3
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.78, n), 20)
    res = run_signed(pp, n, r, keys, np.zeros(0, np.uint64), 21)
    gt = pp.IBLT(n, r, 21)
    gt.insert(_dev(keys))
    out = torch.zeros(len(keys), dtype=torch.int64, device="cuda")
    u = gt.decode(out)
    assert u.rounds == res.rounds and u.recovered_per_round == res.recovered_per_round


@pytest.mark.parametrize("binned", [0, 2], ids=["binned", "direct"])
def test_large_table(pp, binned):
    n, r = 1 << 22, 3
    A, B = _sets(int(0.45 * n), int(0.3 * n), 1 << 20, 22)
    run_signed(pp, n, r, A, B, 23, opts=pp.options(binned=binned))


@pytest.mark.parametrize("binned", [0, 1], ids=["direct", "binned"])
def test_host_loop_and_no_signs(pp, binned):
    n, r = 30000, 4
    A, B = _sets(9000, 9000, 3000, 24)
    a = run_signed(pp, n, r, A, B, 25, opts=pp.options(host_loop=1, binned=binned))
    b = run_signed(pp, n, r, A, B, 25, opts=pp.options(binned=binned), with_signs=False)
    assert a.recovered_per_round == b.recovered_per_round


def test_signed_then_unsigned_on_one_handle(pp):
    """The signed and unsigned decodes share the round bins and the bitmap."""
    n, r = 1 << 21, 3
    A, B = _sets(int(0.4 * n), int(0.3 * n), 1000, 28)
    gt = pp.IBLT(n, r, 29)
    for rep in range(2):
        gt.clear()
        gt.insert(_dev(A))
        gt.delete(_dev(B))
        out = torch.zeros(len(A) + len(B), dtype=torch.int64, device="cuda")
        sg = torch.zeros(len(A) + len(B), dtype=torch.int8, device="cuda")
        res = gt.decode_signed(out, sg)
        assert res.recovered == len(A) + len(B) - 2000 and res.residual_cells == 0
        got = out[: res.recovered].cpu().numpy().view(np.uint64)
        neg = sg[: res.recovered].cpu().numpy() < 0
        assert np.array_equal(np.sort(got[~neg]), np.sort(A[1000:]))
        assert np.array_equal(np.sort(got[neg]), np.sort(B[1000:]))
        gt.clear()
        gt.insert(_dev(A))
        u = gt.decode(torch.zeros(len(A), dtype=torch.int64, device="cuda"))
        assert u.recovered == len(A) and u.residual_cells == 0


@pytest.mark.parametrize("binned", [0, 1], ids=["direct", "binned"])
def test_capacity_error(pp, binned):
    n, r = 20000, 3
    A, B = _sets(6000, 4000, 1000, 26)
    gt = pp.IBLT(n, r, 27, pp.options(binned=binned))
    gt.insert(_dev(A))
    gt.delete(_dev(B))
    out = torch.zeros(100, dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError) as ei:
        gt.decode_signed(out)
    assert ei.value.name == "PP_ERR_CAPACITY"
