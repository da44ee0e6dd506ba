"""Writes full_size.json: the oracle's exact results on the full-size workloads.

Calls only ``oracle`` (and ``ppgen`` for the seeded inputs).  The GPU parity
tests compare the CUDA path against these numbers at sizes where running the
oracle inside the test would take minutes:

* IBLT, 2^26 cells, r=3, load 0.75: rounds, keys recovered per round, cells
  alive per round, and a SHA-256 of each round's sorted key set.
* k-core density sweep, n=2^25, r=4, k=2, c in {0.70,0.76,0.78,0.80,0.85}:
  rounds, s_t, m_t, core sizes, and SHA-256 of the per-vertex and per-edge
  removal rounds (int32 little-endian).

Run from the repository root:  python tests/golden/make_full_size.py
"""
import hashlib
import json
import os
import sys
import time

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import ppgen  # noqa: E402


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def iblt_headline():
    cfg = ppgen.IBLT_HEADLINE
    n, r = cfg["n_cells"], cfg["r"]
    m = ppgen.edges_from_c(cfg["c"], n)
    keys = ppgen.distinct_keys(m, cfg["key_seed"])
    t = oracle.IBLT(n, r, cfg["table_seed"])
    t.insert(keys)
    res = t.decode_rounds()
    rec = [int(k.size) for k in res["keys"]]
    return dict(n_cells=n, r=r, m=m, key_seed=cfg["key_seed"], table_seed=cfg["table_seed"],
                rounds=res["rounds"], recovered_per_round=rec,
                alive_cells_per_round=res["cells_alive"],
                round_sha256=[sha(np.sort(k)) for k in res["keys"]],
                residual_cells=t.residual_cells())


def density_sweep():
    cfg = ppgen.DENSITY_SWEEP
    n, r, k = cfg["n"], cfg["r"], cfg["k"]
    out = []
    for c in cfg["cs"]:
        m = ppgen.edges_from_c(c, n)
        e = ppgen.partitioned_edges(n, r, m, cfg["seed"])
        res = oracle.kcore_rounds(n, k, e)
        out.append(dict(c=c, n=n, r=r, k=k, m=m, seed=cfg["seed"], rounds=res["rounds"],
                        s=res["s"], m_t=res["m"], core_vertices=int((res["vround"] == 0).sum()),
                        core_edges=int((res["eround"] == 0).sum()),
                        vround_sha256=sha(res["vround"].astype("<i4")),
                        eround_sha256=sha(res["eround"].astype("<i4"))))
        print(f"c={c}: {res['rounds']} rounds", file=sys.stderr)
    return out


def main():
    t0 = time.time()
    data = dict(iblt_headline=iblt_headline())
    print(f"iblt done {time.time() - t0:.0f}s", file=sys.stderr)
    data["density_sweep"] = density_sweep()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size.json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    print(f"wrote {path} in {time.time() - t0:.0f}s", file=sys.stderr)


if __name__ == "__main__":
    main()
