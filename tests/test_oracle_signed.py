"""Pins for the signed IBLT recovery (a set difference; Sec. 6 "Motivation")
in the oracle.

A table built by inserting the keys of A and deleting those of B holds the
difference: keys of A \\ B with count contribution +1, keys of B \\ A with -1.
These tests pin ``IBLT.decode_signed`` against:

* the unsigned recovery, on tables with insertions only (every sign +1);
* the set definition: what comes out is exactly A \\ B with sign +1 and
  B \\ A with sign -1 whenever the decode empties the table;
* the swap A <-> B, which flips every sign and nothing else;
* the k = 2 round peel of the hypergraph of A xor B (Sec. 6: recovery is
  peeling at k = 2), round by round.
"""
import numpy as np
import pytest

import oracle
import ppgen


def _table(n, r, seed, A, B):
    t = oracle.IBLT(n, r, seed)
    if len(A):
        t.insert(A)
    if len(B):
        t.insert(B, sign=-1)
    return t


def _sets(n_a, n_b, n_common, seed):
    keys = ppgen.distinct_keys(n_a + n_b + n_common, seed)
    common = keys[:n_common]
    A = np.concatenate([common, keys[n_common:n_common + n_a]])
    B = np.concatenate([common, keys[n_common + n_a:]])
    return A, B, keys[n_common:n_common + n_a], keys[n_common + n_a:]


@pytest.mark.parametrize("n,r,c,seed", [(3000, 3, 0.7, 1), (4096, 4, 0.72, 2), (5000, 3, 0.9, 3)])
def test_insert_only_equals_unsigned(n, r, c, seed):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), 10 + seed)
    a = _table(n, r, seed, keys, [])
    b = a.copy()
    ua = a.decode_rounds()
    sb = b.decode_signed()
    assert sb["rounds"] == ua["rounds"]
    for x, y, sg in zip(ua["keys"], sb["keys"], sb["signs"]):
        assert np.array_equal(np.sort(x), y) and (sg == 1).all()
    assert np.array_equal(a.count, b.count) and np.array_equal(a.keyx, b.keyx)


@pytest.mark.parametrize("n,r,seed", [(4000, 3, 4), (6000, 4, 5), (9000, 3, 6)])
def test_set_difference_recovered(n, r, seed):
    # |A \ B| + |B \ A| = 0.7 n, with many keys in both (they cancel)
    A, B, only_a, only_b = _sets(int(0.45 * n), int(0.25 * n), 3 * n, seed)
    t = _table(n, r, seed, A, B)
    res = t.decode_signed()
    keys = np.concatenate(res["keys"])
    signs = np.concatenate(res["signs"])
    assert np.array_equal(np.sort(keys[signs == 1]), np.sort(only_a))
    assert np.array_equal(np.sort(keys[signs == -1]), np.sort(only_b))
    assert not t.count.any() and not t.keyx.any() and not t.chkx.any()


def test_swap_flips_every_sign():
    n, r, seed = 5000, 3, 7
    A, B, _, _ = _sets(2000, 1500, 4000, 8)
    x = _table(n, r, seed, A, B).decode_signed()
    y = _table(n, r, seed, B, A).decode_signed()
    assert x["rounds"] == y["rounds"]
    for k1, s1, k2, s2 in zip(x["keys"], x["signs"], y["keys"], y["signs"]):
        o1, o2 = np.lexsort((s1, k1)), np.lexsort((-s2, k2))
        assert np.array_equal(k1[o1], k2[o2]) and np.array_equal(s1[o1], -s2[o2])


@pytest.mark.parametrize("n,r,seed,fa,fb", [(4000, 3, 9, 0.4, 0.35), (6000, 4, 10, 0.3, 0.4),
                                            (5000, 3, 11, 0.5, 0.4)])
def test_rounds_equal_the_k2_peel_of_the_difference(n, r, seed, fa, fb):
    A, B, only_a, only_b = _sets(int(fa * n), int(fb * n), n, seed)
    diff = np.concatenate([only_a, only_b])
    cells = oracle.key_cells(n, r, seed, diff).astype(np.uint32)
    ref = oracle.kcore_rounds(n, 2, cells)
    res = _table(n, r, seed, A, B).decode_signed()
    assert res["rounds"] == max([0] + [int(x) for x in ref["eround"]])
    is_a = np.isin(diff, only_a)
    for t in range(1, res["rounds"] + 1):
        sel = ref["eround"] == t
        want = np.sort(diff[sel])
        got_k, got_s = res["keys"][t - 1], res["signs"][t - 1]
        o = np.argsort(got_k)
        assert np.array_equal(got_k[o], want), t
        assert np.array_equal(got_s[o], np.where(is_a[sel][np.argsort(diff[sel])], 1, -1)), t


def test_empty_and_cancelled():
    t = oracle.IBLT(500, 3, 1)
    assert t.decode_signed()["rounds"] == 0
    keys = ppgen.distinct_keys(300, 2)
    t = _table(500, 3, 1, keys, keys)    # everything cancels
    assert not t.count.any() and t.decode_signed()["rounds"] == 0
