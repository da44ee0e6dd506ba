"""CPU: the autotuner's cache (keys, file round trip, applying an entry)."""
import json

import pytest


@pytest.fixture(scope="module")
def tune(ppeel_lib):
    import paper_1302_7014_b300.tune as tune
    return tune


def test_shape_key_buckets(tune):
    k = tune.shape_key("NVIDIA B300", [4, 3, 3], 470_000_000, 4096)
    assert k == "NVIDIA B300|r=3/4|cells=2^29|tables=2^12"
    assert tune.shape_key("G", [3], 1 << 20, 1) == "G|r=3|cells=2^20|tables=2^0"
    # sizes within a factor sqrt(2) share a bucket
    assert tune.shape_key("G", [3], int(1.3 * (1 << 20)), 100) == tune.shape_key("G", [3], 1 << 20, 128)


def test_store_and_load(tune, tmp_path):
    p = str(tmp_path / "sub" / "t.json")
    assert tune.load_cache(p) == {}
    tune.store("a", {"ctas_per_sm": 4, "apply_ctas": 2, "binned": 1, "insert_chunk": 4096}, p, best_ms=1.5)
    tune.store("b", {"ctas_per_sm": 8, "apply_ctas": 3, "binned": 2, "insert_chunk": 1024}, p)
    data = json.load(open(p))
    assert data["a"]["options"]["apply_ctas"] == 2 and data["a"]["best_ms"] == 1.5
    assert tune.load_cache(p)["b"]["options"]["binned"] == 2
    (tmp_path / "bad.json").write_text("{not json")
    assert tune.load_cache(str(tmp_path / "bad.json")) == {}


def test_options_from_entry(tune):
    import paper_1302_7014_b300 as pp
    base = pp.options(max_rounds=77, stats_rounds=9)
    o = tune.options_from(base, {"ctas_per_sm": 2, "apply_ctas": 4, "binned": 2, "insert_chunk": 16384})
    assert (o.ctas_per_sm, o.apply_ctas, o.binned, o.insert_chunk) == (2, 4, 2, 16384)
    assert (o.max_rounds, o.stats_rounds) == (77, 9)   # untouched fields
    d = pp.options()
    assert (d.apply_ctas, d.frontier_switch, d.insert_chunk) == (3, 2, 4096)
