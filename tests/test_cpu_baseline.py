"""CPU: the OpenMP round simulator (the all-cores CPU baseline) against the
oracle -- the same keys per round, the same rounds and the same residue --
with one thread and with every core."""
import numpy as np
import pytest

import cpu_baseline as cb
import oracle
import ppgen


@pytest.mark.parametrize("n,r,c,seed", [(30011, 3, 0.75, 1), (50000, 4, 0.7, 2), (20000, 3, 0.9, 3),
                                        (9000, 2, 0.4, 4), (7001, 5, 0.6, 5), (4096, 4, 0.85, 6)])
@pytest.mark.parametrize("threads", [1, 0], ids=["1-thread", "all-cores"])
def test_omp_rounds_equal_oracle(n, r, c, seed, threads):
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n), seed + 50)
    got = cb.build_and_decode(n, r, seed, keys, n_threads=threads)
    t = oracle.IBLT(n, r, seed)
    t.insert(keys)
    res = t.decode_rounds()
    assert got["status"] == 0 and got["rounds"] == res["rounds"]
    for a, b in zip(got["keys"], res["keys"]):
        assert (np.sort(a) == b).all()
    assert (got["count"] == t.count).all() and (got["keyx"] == t.keyx).all() and (got["chkx"] == t.chkx).all()


def test_omp_round_limit_and_empty():
    keys = ppgen.distinct_keys(ppgen.edges_from_c(0.8, 20000), 9)
    got = cb.build_and_decode(20000, 3, 9, keys, max_rounds=3)
    t = oracle.IBLT(20000, 3, 9)
    t.insert(keys)
    res = t.decode_rounds(max_rounds=3)
    assert got["status"] == oracle.ROUND_LIMIT and got["rounds"] == 3
    assert (got["count"] == t.count).all() and (got["keyx"] == t.keyx).all()
    e = cb.build_and_decode(100, 3, 1, np.zeros(0, np.uint64))
    assert e["rounds"] == 0 and e["status"] == 0
