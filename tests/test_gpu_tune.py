"""GPU: the batched engine's autotuner (pp_tune_batch).  Every candidate it
times must reproduce the untuned per-table results, and the batch decoded with
the options it picks must equal the CPU oracle, table by table."""
import numpy as np
import pytest

import ppgen
from test_gpu_batch import _specs, check_against_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods(ppeel_lib):
    import paper_1302_7014_b300 as pp
    import paper_1302_7014_b300.batch as batch
    import paper_1302_7014_b300.tune as tune
    return pp, batch, tune


def _inputs(specs):
    keys = [ppgen.distinct_keys(ppgen.edges_from_c(s[2], s[0]), s[4]) for s in specs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    dk = torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda()
    out = torch.full((int(koff[-1]),), -1, dtype=torch.int64, device="cuda")
    return keys, koff, dk, out


@pytest.mark.parametrize("rs", [(3,), (3, 4), (2, 5)], ids=["r3", "r3-4", "r2-5"])
def test_tuned_batch_matches_oracle(mods, tmp_path, rs):
    pp, bm, tune = mods
    specs = _specs(48, 7 + len(rs), rs=rs, lo=8, hi=15, c_lo=0.5, c_hi=0.95)
    keys, koff, dk, out = _inputs(specs)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs])
    cache = str(tmp_path / "tune.json")
    res = tune.tune_batch(b, dk, koff, out, koff, reps=1, path=cache)
    assert res.mismatches == 0 and not res.from_cache
    assert len(res.candidates_ms) >= 10 and min(res.candidates_ms) > 0
    assert res.best_ms <= res.default_ms + 1e-6
    o = b.options()
    assert {k: int(getattr(o, k)) for k in tune.TUNED_FIELDS} == res.options
    # decode with the tuned options, against the oracle
    b.build(dk, koff)
    out.fill_(-1)
    r2 = b.decode(out, koff)
    check_against_oracle(specs, keys, koff, r2, out.cpu().numpy().view(np.uint64), b, cells_every=7)
    # a second batch of the same shape takes the cached options without searching
    b2 = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs])
    hit = tune.tune_batch(b2, dk, koff, out, koff, reps=1, path=cache)
    assert hit.from_cache and hit.options == res.options
    o2 = b2.options()
    assert {k: int(getattr(o2, k)) for k in tune.TUNED_FIELDS} == res.options
    b2.build(dk, koff)
    out.fill_(-1)
    r3 = b2.decode(out, koff)
    check_against_oracle(specs, keys, koff, r3, out.cpu().numpy().view(np.uint64))
    b.close()
    b2.close()


def test_set_options_keeps_results(mods):
    pp, bm, tune = mods
    specs = _specs(40, 3, rs=(3, 4), lo=8, hi=16, c_lo=0.6, c_hi=1.0)
    keys, koff, dk, out = _inputs(specs)
    b = bm.Batch([s[0] for s in specs], [s[1] for s in specs], [s[3] for s in specs])
    for o in (pp.options(binned=2, insert_chunk=512, ctas_per_sm=1),
              pp.options(binned=1, apply_ctas=2, ctas_per_sm=8, rounds=1),
              pp.options(rounds=2, insert_chunk=1024), pp.options()):
        b.set_options(o)
        b.build(dk, koff)
        out.fill_(-1)
        res = b.decode(out, koff)
        check_against_oracle(specs, keys, koff, res, out.cpu().numpy().view(np.uint64))
    b.close()
