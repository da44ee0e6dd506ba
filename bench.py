"""Benchmark: IBLT build + round-synchronous decode, 2^26 cells, r = 3, load 0.75.

One step = clear the table, insert m = 0.75 * 2^26 keys (build), decode it by
round-synchronous peeling until the frontier is empty (initial scan, rounds,
termination).  ``value`` = keys recovered per second of the whole step, with
the keys already in HBM; ``e2e`` = the same through the public API with the
keys uploaded from pinned host memory and the recovered keys read back to host
memory inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank decodes its own table (independent
problems, weak scaling); the slowest rank's time counts.  ``--impl reference``
times the CPU oracle (the only other place this file runs ``oracle/``) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ppgen  # noqa: E402

METRIC = "keys recovered/s & peel ms at n=2^26 r=3 c=0.75; batched vs plain; p99 ms"
UNIT = "keys/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6400.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources the headline table's build and decode are compiled from (the
# k-core, batch and server files do not reach those kernels).
HEADLINE_SOURCES = ("common.cu", "device.cuh", "host.cuh", "iblt.cu", "iblt_binned.cuh", "iblt_kernels.cuh",
                    "iblt_rounds.cuh", "iblt_tiles.cuh", "iblt_trounds.cuh", "iblt_types.cuh", "tiles.cu")


def csrc_digest() -> str:
    """Digest of the headline sources' code: line comments and blank lines are
    left out, so that a comment edit does not void the stored traffic."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1302_7014_b300", "csrc")
    for name in HEADLINE_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            lines = (ln.split(b"//", 1)[0].rstrip() for ln in f.read().splitlines())
            h.update(name.encode() + b"\n".join(ln for ln in lines if ln))
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernels
    have not changed since it was taken."""
    try:
        with open(TRAFFIC_PATH) as f:
            t = json.load(f)
        e = t.get(kernel)
        if e and e.get("csrc_digest") == csrc_digest():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before
    the warm-up; stop() keeps the samples stamped inside the timed region
    (wall clock), or the two nearest ones when the region is shorter than the
    sampling period."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ppeel_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0: float, t1: float):
        """Samples between wall-clock times t0 and t1 (time.time())."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        import datetime
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(p[2]), float(p[3]), p[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [x for x in rows if t0 <= x[0] <= t1]
        window = "timed region"
        if not inside:
            inside = sorted(rows, key=lambda x: min(abs(x[0] - t0), abs(x[0] - t1)))[:2]
            window = "nearest samples"
        reasons = sorted({n for x in inside for n, v in zip(self.REASONS, x[3]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median([x[1] for x in inside])), "sm_max_mhz": max(x[2] for x in inside),
                "reasons": reasons, "samples": len(inside), "window": window}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_workload(cfg, rank: int):
    """(key seed, table seed) of this rank's replica: every rank decodes its own
    table of the same shape with its own keys (weak scaling, no exchange)."""
    return cfg["key_seed"] + 7919 * rank, cfg["table_seed"] + rank


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time: the slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: int, dist, device) -> int:
    """Units processed by the whole job."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def oracle_sample(n_cells: int, r: int, c: float, key_seed: int, table_seed: int):
    """Build + round-synchronous decode of one table with the CPU oracle.
    Returns (keys recovered, seconds)."""
    import oracle
    keys = ppgen.distinct_keys(ppgen.edges_from_c(c, n_cells), key_seed)
    t0 = time.perf_counter()
    t = oracle.IBLT(n_cells, r, table_seed)
    t.insert(keys)
    res = t.decode_rounds()
    dt = time.perf_counter() - t0
    return int(sum(k.size for k in res["keys"])), dt


def cpu_baseline(cfg):
    """The oracle as it stands, single thread, on 2^22-cell tables of the same
    recipe: one table per key seed until about 10 s of CPU time (12 at most)."""
    n = 1 << 22
    total, secs, k = 0, 0.0, 0
    while k < 12 and secs < 10.0:
        got, dt = oracle_sample(n, cfg["r"], cfg["c"], cfg["key_seed"] + 200 + k, cfg["table_seed"])
        total, secs, k = total + got, secs + dt, k + 1
    out = {"value": total / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{k} x one build + round-synchronous decode of a 2^22-cell table, r=3, "
                     f"load 0.75 ({total} keys, {secs:.1f} s)"}
    try:
        out["all_cores"] = cpu_all_cores(cfg)
    except Exception as exc:  # informative only
        out["all_cores"] = {"error": str(exc)}
    return out


def cpu_all_cores(cfg):
    """The OpenMP round simulator (cpu_baseline/rounds_omp.c, checked against
    the oracle in the tests) on every host core: one build + decode of the full
    headline table, the same keys as the GPU's."""
    import cpu_baseline as cb
    cores = os.cpu_count() or 1
    n = cfg["n_cells"]
    keys = ppgen.distinct_keys(ppgen.edges_from_c(cfg["c"], n), cfg["key_seed"])
    cb.build_and_decode(1 << 16, cfg["r"], cfg["table_seed"], keys[: 1 << 15], n_threads=cores)  # warm-up
    res = cb.build_and_decode(n, cfg["r"], cfg["table_seed"], keys, n_threads=cores)
    got = int(sum(k.size for k in res["keys"]))
    secs = res["build_s"] + res["decode_s"]
    return {"value": got / secs, "unit": UNIT, "cores": cores, "threads": cb.threads(),
            "kind": "openmp round simulator", "build_s": res["build_s"], "decode_s": res["decode_s"],
            "rounds": res["rounds"],
            "sample": f"one build + round-synchronous decode of the full 2^{int(np.log2(n))}-cell table, "
                      f"r={cfg['r']}, load {cfg['c']} ({got} keys, {secs:.1f} s)"}


def run_reference(args, cfg):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    n = 1 << 21
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(n, cfg["r"], cfg["c"], cfg["key_seed"] + 1, cfg["table_seed"])
    total, secs = 0, 0.0
    for s in range(args.steps):
        got, dt = oracle_sample(n, cfg["r"], cfg["c"], cfg["key_seed"] + 100 + s, cfg["table_seed"])
        total += got
        secs += dt
    v = total / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "sample_cells": n, "r": cfg["r"], "load": cfg["c"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} x build + round-synchronous decode of a "
                                       f"2^21-cell table, r=3, load 0.75"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batched(pp, torch, args):
    """4096 IBLTs (cells log-uniform in [2^8, 2^20), r in {3, 4}, load uniform in
    [0.5, 0.9 c*]): one batched graph launch vs a loop of plain per-table decodes,
    same tables, same keys, identical output."""
    import paper_1302_7014_b300.batch as pb
    tabs = ppgen.batch_tables(4096)
    keys = [t.keys() for t in tabs]
    koff = np.concatenate([[0], np.cumsum([k.size for k in keys])]).astype(np.uint64)
    total_keys = int(koff[-1])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dkeys = torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda()
        out = torch.empty(total_keys, dtype=torch.int64, device="cuda")
    stream.synchronize()
    b = pb.Batch([t.n_cells for t in tabs], [t.r for t in tabs], [t.table_seed for t in tabs])

    def bstep():
        # clear + insert + decode in one pp_batch_build_decode (the build's
        # write-out finds F_1)
        return b.build_decode(dkeys, koff, out, koff, stream=stream)

    steps = max(3, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        for _ in range(max(2, args.warmup)):
            res = bstep()
        torch.cuda.synchronize()
        e0.record(stream)
        rec = 0
        for _ in range(steps):
            res = bstep()
            rec += int(res.recovered.sum())
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / steps, rec, res

    d_ms, rec, res = timed()   # default options
    d_rec = res.recovered.copy()
    # the project's autotuner picks the run-time knobs on this batch (its own
    # search times each candidate; the winner is then timed like the default)
    import paper_1302_7014_b300.tune as pt
    tuned = pt.tune_batch(b, dkeys, koff, out, koff, reps=2, use_cache=False, stream=stream)
    b_ms, rec, res = timed()
    b_rounds = int(res.rounds.max())
    b_rec = res.recovered.copy()
    tuned_identical = bool((b_rec == d_rec).all())
    b.close()
    del out
    torch.cuda.empty_cache()
    # plain loop: one handle per table, created before timing
    handles = [pp.IBLT(t.n_cells, t.r, t.table_seed) for t in tabs]
    with torch.cuda.stream(stream):
        out = torch.empty(total_keys, dtype=torch.int64, device="cuda")
    stream.synchronize()
    views = [(dkeys[int(koff[i]):int(koff[i + 1])], out[int(koff[i]):int(koff[i + 1])] if koff[i + 1] > koff[i]
              else out[:1]) for i in range(len(tabs))]

    def pstep():
        got = []
        for h, (kv, ov) in zip(handles, views):
            h.clear(stream)
            h.insert(kv, stream)
            got.append(h.decode(ov, stream=stream).recovered)
        return got

    pstep()
    torch.cuda.synchronize()
    psteps = 2
    e0.record(stream)
    for _ in range(psteps):
        got = pstep()
    e1.record(stream)
    stream.synchronize()
    p_ms = e0.elapsed_time(e1) / psteps
    identical = bool((np.array(got) == b_rec).all())
    for h in handles:
        h.close()
    del out, dkeys
    torch.cuda.empty_cache()
    n = len(tabs)
    # sector-floor bytes of one step, as for the headline table: the clear writes
    # every 32 B cell, the build 8 + 64 r B per key, the rounds 64 r + 16 B per
    # key (no scan: the build's write-out finds F_1); the arena is far larger
    # than L2
    cells = sum(t.n_cells for t in tabs)
    step_bytes = 32 * cells + sum(k.size * (8 + 64 * t.r) for k, t in zip(keys, tabs)) + \
        sum(k.size * (64 * t.r + 16) for k, t in zip(keys, tabs))
    peak, peak_kind = hbm_peak()
    achieved = step_bytes / (b_ms * 1e-3) / 1e9
    return {"workload": "4096 IBLTs, cells log-uniform [2^8,2^20), r in {3,4}, load U[0.5, 0.9 c*]",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                         "model": "sector floor: 32 B/cell clear + (8+64r) B/key build + (64r+16) B/key "
                                  "rounds"},
            "tables": n, "cells": int(sum(t.n_cells for t in tabs)), "keys": total_keys,
            "batched_ms": b_ms, "plain_loop_ms": p_ms,
            "batched_tables_per_s": n / (b_ms * 1e-3), "plain_tables_per_s": n / (p_ms * 1e-3),
            "autotuned": {"options": tuned.options, "default_ms": d_ms, "tuned_ms": b_ms,
                          "default_tables_per_s": n / (d_ms * 1e-3), "tuned_tables_per_s": n / (b_ms * 1e-3),
                          "candidates": len(tuned.candidates_ms), "search_ms": tuned.candidates_ms,
                          "identical_output": tuned_identical,
                          "key": tuned.key},
            "batched_keys_per_s": rec / steps / (b_ms * 1e-3), "speedup": p_ms / b_ms,
            "rounds_max": b_rounds, "identical_output": identical,
            "step": "one pp_batch_build_decode: clear + insert + decode of every table"}


def _serve_stream(ps, srv, reqs):
    """Submit reqs open loop at their scheduled arrival times; (latencies s, keys, span s)."""
    t0 = ps.server_now() + 0.01
    tickets = []
    for at, spec in reqs:
        while ps.server_now() < t0 + at:
            pass
        tickets.append(srv.submit(spec.n_cells, 3, spec.table_seed, spec.m, key_seed=spec.key_seed,
                                  arrival_s=t0 + at))
    lat, keys, last = [], 0, t0
    for t in tickets:
        r = srv.wait(t, 600.0)
        lat.append(r["done_s"] - r["arrival_s"])
        keys += r["recovered"]
        last = max(last, r["done_s"])
    return np.array(lat), keys, last - t0


def bench_served(pp, torch, args):
    """Open-loop Poisson arrivals (mean 20k req/s) of decode requests, cells
    log-uniform in [2^10, 2^22), r = 3, load U[0.6, 0.8]; keys generated on the
    device from each request's seed.  Latency = completion - scheduled arrival.
    When 20k req/s exceeds what the server sustains, its latencies are queueing
    delay; a second stream at 70 % of the measured capacity gives the latency
    of the service itself."""
    import paper_1302_7014_b300.server as ps
    rate = 20000.0
    n_req = max(1, int(rate * args.serve_seconds))
    reqs = ppgen.serving_requests(n_req, rate_per_s=rate)
    srv = ps.Server(arena_cells=1 << 29, arena_keys=1 << 29, max_slots=8192, r=3)
    # warm up the kernels
    for at, spec in reqs[:4]:
        srv.wait(srv.submit(spec.n_cells, 3, spec.table_seed, spec.m, key_seed=spec.key_seed), 120.0)
    it0 = srv.stats()["iterations"]
    lat, keys, span = _serve_stream(ps, srv, reqs)
    iters = srv.stats()["iterations"] - it0
    served_rate = n_req / span
    out = {"workload": "Poisson 20k req/s, cells log-uniform [2^10,2^22), r=3, load U[0.6,0.8]",
           "requests": n_req, "arrival_window_s": args.serve_seconds, "span_s": span,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "keys_per_s": keys / span, "requests_per_s": served_rate,
           "offered_req_per_s": rate, "saturated": bool(served_rate < 0.95 * rate),
           "iterations": iters, "keys_source": "generated on the device from request seeds"}
    if out["saturated"]:
        rate2 = 0.7 * served_rate
        n2 = max(1, int(rate2 * args.serve_below_seconds))
        lat2, keys2, span2 = _serve_stream(ps, srv, ppgen.serving_requests(n2, rate_per_s=rate2, seed=6))
        out["below_capacity"] = {
            "offered_req_per_s": rate2, "requests": n2, "arrival_window_s": args.serve_below_seconds,
            "span_s": span2, "requests_per_s": n2 / span2,
            "p50_ms": float(np.percentile(lat2, 50) * 1e3), "p99_ms": float(np.percentile(lat2, 99) * 1e3),
            "keys_per_s": keys2 / span2, "note": "same request mix, 70 % of the capacity measured above"}
    srv.stop()
    return out


def bench_served_vs_plain(pp, torch, args, k=1000):
    """The first k requests of the served mix (Poisson stream seed 5, cells
    log-uniform in [2^10, 2^22), r = 3, load U[0.6, 0.8]) two ways: a plain loop
    of per-request build + decode calls, one handle per request made and keys
    uploaded before timing; and the server, every request submitted at once
    (keys generated on the device from their seeds, inside the served time).
    Tables/s of each, and the per-request rounds and recovered counts compared."""
    import paper_1302_7014_b300.server as ps
    specs = [s for _, s in ppgen.serving_requests(k, rate_per_s=20000.0)]
    stream = torch.cuda.Stream()
    handles = [pp.IBLT(s.n_cells, 3, s.table_seed) for s in specs]
    with torch.cuda.stream(stream):
        keys = [torch.from_numpy(s.keys().view(np.int64)).cuda() for s in specs]
        outs = [torch.empty(max(1, s.m), dtype=torch.int64, device="cuda") for s in specs]
    stream.synchronize()
    for h, kk, o in list(zip(handles, keys, outs))[:20]:   # warm-up: graphs, workspaces
        h.build(kk, stream)
        h.decode(o, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    plain = []
    for h, kk, o in zip(handles, keys, outs):
        h.build(kk, stream)
        res = h.decode(o, stream=stream)
        plain.append((res.rounds, res.recovered))
    ev[1].record(stream)
    stream.synchronize()
    p_s = ev[0].elapsed_time(ev[1]) * 1e-3
    for h in handles:
        h.close()
    del keys, outs
    torch.cuda.empty_cache()
    srv = ps.Server(arena_cells=1 << 29, arena_keys=1 << 29, max_slots=8192, r=3)
    for s in specs[:4]:
        srv.wait(srv.submit(s.n_cells, 3, s.table_seed, s.m, key_seed=s.key_seed), 120.0)
    t0 = ps.server_now()
    tickets = [srv.submit(s.n_cells, 3, s.table_seed, s.m, key_seed=s.key_seed, arrival_s=t0) for s in specs]
    served = []
    last = t0
    for t in tickets:
        r = srv.wait(t, 600.0)
        served.append((r["rounds"], r["recovered"]))
        last = max(last, r["done_s"])
    srv.stop()
    s_s = last - t0
    return {"workload": f"first {k} requests of the served mix (cells log-uniform [2^10,2^22), r=3, "
                        "load U[0.6,0.8]), all at once",
            "plain_loop_s": p_s, "served_s": s_s, "plain_tables_per_s": k / p_s, "served_tables_per_s": k / s_s,
            "speedup": p_s / s_s, "identical_output": plain == served,
            "plain": "per request pp_iblt_build + pp_iblt_decode on its own handle (made before timing), "
                     "keys on the device before timing",
            "served": "pp_server_submit of every request at t0, keys generated on the device in the served time"}


def bench_subrounds(pp, torch, table, dkeys, out, stream, m, steps):
    """The headline table decoded in the paper's own order: one sub-table per
    sub-round (Sec. 6 "Implementation Details", App. B), same build."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    table.build(dkeys, stream)
    res = table.decode_subrounds(out, stream=stream)
    assert res.recovered == m and res.residual_cells == 0
    ms = []
    for _ in range(steps):
        table.build(dkeys, stream)
        ev[0].record(stream)
        res = table.decode_subrounds(out, stream=stream)
        ev[1].record(stream)
        stream.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
    d = float(np.mean(ms))
    return {"workload": "headline table, one sub-table per sub-round", "decode_ms": d,
            "decode_keys_per_s": res.recovered / (d * 1e-3), "subrounds": res.rounds,
            "recovered_per_subround_first": res.recovered_per_round[:6]}


def bench_signed(pp, torch, args):
    """Sparse recovery (Sec. 6 "Motivation"): 2^26 cells hold the difference of
    two key sets, 0.45 n keys only in A and 0.30 n only in B (plus 0.25 n in
    both, which cancel); decode_signed recovers A \\ B with sign +1 and B \\ A
    with sign -1."""
    n, r = 1 << 26, 3
    na, nb, nc = int(0.45 * n), int(0.30 * n), int(0.25 * n)
    keys = ppgen.distinct_keys(na + nb + nc, 31)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dk = torch.from_numpy(keys.view(np.int64)).cuda()
        out = torch.empty(na + nb, dtype=torch.int64, device="cuda")
        sg = torch.empty(na + nb, dtype=torch.int8, device="cuda")
    stream.synchronize()
    t = pp.IBLT(n, r, 0x5195)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ms = []
    for it in range(3 + max(3, min(args.steps, 5))):
        t.build(dk[:nc + na], stream)               # A = common + only-A
        t.delete(dk[:nc], stream)                   # B = common + only-B
        t.delete(dk[nc + na:], stream)
        ev[0].record(stream)
        res = t.decode_signed(out, sg, stream=stream)
        ev[1].record(stream)
        stream.synchronize()
        if it >= 3:
            ms.append(ev[0].elapsed_time(ev[1]))
    neg = int((sg[: res.recovered] < 0).sum().item())
    assert res.recovered == na + nb and neg == nb and res.residual_cells == 0
    d = float(np.mean(ms))
    t.close()
    del dk, out, sg
    torch.cuda.empty_cache()
    return {"workload": "2^26 cells, r=3: |A \\ B| = 0.45 n, |B \\ A| = 0.30 n, |A & B| = 0.25 n",
            "decode_ms": d, "keys_per_s": res.recovered / (d * 1e-3), "rounds": res.rounds,
            "recovered_plus": res.recovered - neg, "recovered_minus": neg}


def bench_scatter(pp, torch, n_log2=26, m=6_900_000, reps=5):
    """The GPU's rate for the decode's access pattern: m distinct random 32-byte
    cells of a 2^26-cell (2 GB) table read and written back, read only, or
    overwritten only (pp_probe_scatter), in random order and sorted by
    4096-cell tile (the order the tile rounds apply them in).  m is the number
    of cells a middle round of the headline decode touches."""
    import ctypes
    from paper_1302_7014_b300 import _lib
    lib = _lib.load()
    n = 1 << n_log2
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        cells = torch.zeros(n * 32, dtype=torch.uint8, device="cuda")
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        idx = torch.randperm(n, device="cuda", generator=g)[:m].to(torch.int32)
        by_tile = torch.sort(idx)[0]   # cell order is also tile order
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sp = ctypes.c_void_p(stream.cuda_stream)
    out = {}
    for order, ix in (("random", idx), ("tile_sorted", by_tile)):
        for mode, name in ((0, "read_write"), (1, "read"), (2, "write")):
            ts = []
            for rep in range(reps + 1):
                with torch.cuda.stream(stream):
                    flush.fill_(rep)   # the table is 16x L2; this also clears the previous pass's lines
                ev[0].record(stream)
                st = lib.pp_probe_scatter(ctypes.c_void_p(cells.data_ptr()), n, ctypes.c_void_p(ix.data_ptr()),
                                          m, mode, sp)
                ev[1].record(stream)
                stream.synchronize()
                if st != 0:
                    raise RuntimeError(lib.pp_last_error().decode())
                if rep:
                    ts.append(ev[0].elapsed_time(ev[1]))
            ms = float(np.median(ts))
            acc = m * (2 if mode == 0 else 1)
            out[f"{order}_{name}"] = {"ms": ms, "accesses_per_s": acc / (ms * 1e-3)}
    del cells, idx, by_tile, flush
    torch.cuda.empty_cache()
    return {"workload": f"{m} distinct random 32 B cells of a 2^{n_log2}-cell table", **out}


def bench_kcore(pp, torch, args):
    """k-core peeling of the density sweep (n = 2^25 vertices in 4 parts, r = 4,
    k = 2, one vertex per part per edge): the whole call (incidence build +
    rounds) in full rounds and in sub-rounds."""
    cfg = ppgen.DENSITY_SWEEP
    n, r, k = cfg["n"], cfg["r"], cfg["k"]
    off = [int(x) for x in np.asarray(ppgen.part_offsets(n, r))]
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    rows = []
    for c in cfg["cs"]:
        m = ppgen.edges_from_c(c, n)
        e = ppgen.partitioned_edges(n, r, m, cfg["seed"])
        with torch.cuda.stream(stream):
            d = torch.from_numpy(e.view(np.int32)).cuda()
        stream.synchronize()
        del e

        def timed(fn, reps=3):
            fn()
            best = []
            for _ in range(reps):
                ev[0].record(stream)
                res = fn()
                ev[1].record(stream)
                stream.synchronize()
                best.append(ev[0].elapsed_time(ev[1]))
            return res, float(np.median(best))

        full, full_ms = timed(lambda: pp.peel_kcore(n, r, k, d, stream=stream))
        # the same call writing every vertex's and every edge's removal round
        with torch.cuda.stream(stream):
            vr = torch.empty(n, dtype=torch.int32, device="cuda")
            er = torch.empty(m, dtype=torch.int32, device="cuda")
        _, out_ms = timed(lambda: pp.peel_kcore(n, r, k, d, vr, er, stream=stream))
        del vr, er
        sub, sub_ms = timed(lambda: pp.peel_kcore_subrounds(n, r, k, d, off, stream=stream, round_cap=1 << 14))
        # sector-floor bytes of the call: per removed edge its alive-flag sector
        # RMW (64 B), its row (one 32 B sector), r degree sector RMWs (64 r B) and
        # its r incidences (4 r B); per incidence of the CSR build one random
        # degree atomic (a 64 B sector RMW) and one 4 B scatter write
        removed = m - int(full.core_edges)
        model = removed * (64 + 32 + 64 * r + 4 * r) + m * r * (64 + 4)
        peak, _ = hbm_peak()
        achieved = model / (full_ms * 1e-3) / 1e9
        rows.append({"c": c, "edges": m, "rounds": full.rounds, "core_vertices": full.core_vertices,
                     "core_edges": full.core_edges, "ms": full_ms, "edges_per_s": m / (full_ms * 1e-3),
                     "model_bytes": model, "achieved_gbs": achieved, "frac": achieved / peak,
                     "ms_with_round_outputs": out_ms,
                     "subrounds": sub.rounds, "subround_ms": sub_ms,
                     "same_core": bool(sub.core_vertices == full.core_vertices
                                       and sub.core_edges == full.core_edges)})
        del d
        torch.cuda.empty_cache()
    # the plain-peel configuration: 2^14 vertices (microseconds)
    pc = ppgen.PLAIN_PEEL
    pe = ppgen.partitioned_edges(pc["n"], pc["r"], ppgen.edges_from_c(pc["c"], pc["n"]), pc["seed"])
    with torch.cuda.stream(stream):
        pd = torch.from_numpy(pe.view(np.int32)).cuda()
    stream.synchronize()
    for _ in range(5):
        pres = pp.peel_kcore(pc["n"], pc["r"], pc["k"], pd, stream=stream)
    us = []
    for _ in range(50):
        ev[0].record(stream)
        pres = pp.peel_kcore(pc["n"], pc["r"], pc["k"], pd, stream=stream)
        ev[1].record(stream)
        stream.synchronize()
        us.append(ev[0].elapsed_time(ev[1]) * 1e3)
    plain = {"workload": "plain peel n=2^14 r=3 k=2 c=0.7 (%d edges)" % pe.shape[0], "rounds": pres.rounds,
             "core_vertices": pres.core_vertices, "us_median": float(np.median(us)),
             "us_p10": float(np.percentile(us, 10)), "us_p90": float(np.percentile(us, 90)),
             "timed": "one pp_peel_kcore call (automatic mode: every round inside one thread block)"}
    return {"workload": cfg["name"], "k": k, "parts": r,
            "roofline_model": "sector floor per removed edge 64 (alive flag) + 32 (row) + 64 r (degrees) + 4 r "
                              "(incidences) B, plus per incidence of the CSR build 64 (degree atomic) + 4 "
                              "(scatter) B; frac of the measured HBM copy bandwidth",
            "timed": "one pp_peel_kcore call: degree histogram, then edge-centric rounds while the frontier "
                     "is at least half the edges left, incidence lists for the edges left and "
                     "vertex-centric rounds after that; 'ms' returns the statistics and the core, "
                     "'ms_with_round_outputs' also writes every vertex's and edge's removal round",
            "densities": rows, "plain_peel": plain}


def bench_tables(pp, torch, args):
    """Table 1 (rounds of G^4_{n,cn}, k = 2) and Table 5 (sub-rounds with 4
    sub-tables) at n = 10^4, 1000 trials per density, each density one peel of
    the trials' disjoint union (10^7 vertices)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    n, r, trials = 10000, 4, 1000
    out = {"workload": "n=10^4, r=4, k=2, 1000 trials per density as one disjoint union",
           "table1": [], "table5": []}
    for name, kind, cs in (("table1", "distinct", (0.70, 0.75, 0.80, 0.85)),
                           ("table5", "partitioned", (0.70, 0.75))):
        for c in cs:
            e, uoff, to_trials = ppgen.trials_union(n, r, ppgen.edges_from_c(c, n), trials, 7, kind)
            d = torch.from_numpy(e.view(np.int32)).cuda()
            vr = torch.empty(n * trials, dtype=torch.int32, device="cuda")

            def run():
                if uoff is None:
                    return pp.peel_kcore(n * trials, r, 2, d, vr, round_cap=1 << 12)
                return pp.peel_kcore_subrounds(n * trials, r, 2, d, uoff, vr, round_cap=1 << 12)
            run()
            torch.cuda.synchronize()
            ev[0].record()
            run()
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1])
            per = to_trials(vr.cpu().numpy())
            rounds = per.max(axis=1)
            out[name].append({"c": c, "mean_rounds": float(rounds.mean()),
                              "failed": int((per == 0).any(axis=1).sum()), "ms": ms,
                              "trials_per_s": trials / (ms * 1e-3)})
            del d, vr
    torch.cuda.empty_cache()
    return out


def profile_case(pp, torch, args, cfg):
    """One call of a secondary workload, two warm-up calls before it, for a
    profiler's launch list or capture (--host-loop drives its rounds from the
    host, which ncu needs to see the round kernels one by one)."""
    opts = pp.options(host_loop=1 if args.host_loop else 0)
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    if args.profile_case == "served":
        # a burst of 2000 requests of the served mix, submitted at once
        import paper_1302_7014_b300.server as ps
        srv = ps.Server(arena_cells=1 << 29, arena_keys=1 << 29, max_slots=8192, r=3)
        reqs = ppgen.serving_requests(2000)
        for at, spec in reqs[:4]:
            srv.wait(srv.submit(spec.n_cells, 3, spec.table_seed, spec.m, key_seed=spec.key_seed), 120.0)
        st0 = srv.stats()
        t0 = time.time()
        tickets = [srv.submit(spec.n_cells, 3, spec.table_seed, spec.m, key_seed=spec.key_seed) for _, spec in reqs]
        keys = sum(srv.wait(t, 600.0)["recovered"] for t in tickets)
        dt = time.time() - t0
        st = srv.stats()
        its = st["iterations"] - st0["iterations"]
        it_us = st["iteration_us"] - st0["iteration_us"]
        srv.stop()
        print(json.dumps({"profile_case": "served", "requests": len(reqs), "s": dt, "keys_per_s": keys / dt,
                          "iterations": its, "ms_per_iteration": dt * 1e3 / max(its, 1),
                          "gpu_wait_share": (st["gpu_wait_us"] - st0["gpu_wait_us"]) / max(it_us, 1)}))
        return
    if args.profile_case == "kcore":
        sw = ppgen.DENSITY_SWEEP
        n, r, k = sw["n"], sw["r"], sw["k"]
        e = ppgen.partitioned_edges(n, r, ppgen.edges_from_c(args.profile_c, n), sw["seed"])
        d = torch.from_numpy(e.view(np.int32)).cuda()
        call = lambda: pp.peel_kcore(n, r, k, d, opts=opts, stream=stream)
        what = f"pp_peel_kcore, {sw['name']}, c={args.profile_c}"
    elif args.profile_case == "plain":
        pc = ppgen.PLAIN_PEEL
        e = ppgen.partitioned_edges(pc["n"], pc["r"], ppgen.edges_from_c(pc["c"], pc["n"]), pc["seed"])
        d = torch.from_numpy(e.view(np.int32)).cuda()
        call = lambda: pp.peel_kcore(pc["n"], pc["r"], pc["k"], d, opts=opts, stream=stream)
        what = "pp_peel_kcore, plain peel n=2^14 r=3 k=2 c=0.7"
    elif args.profile_case == "batched":
        import paper_1302_7014_b300.batch as pb
        tabs = ppgen.batch_tables(4096)
        keys = [t.keys() for t in tabs]
        koff = np.concatenate([[0], np.cumsum([x.size for x in keys])]).astype(np.uint64)
        dk = torch.from_numpy(np.concatenate(keys).view(np.int64)).cuda()
        out = torch.empty(int(koff[-1]), dtype=torch.int64, device="cuda")
        b = pb.Batch([t.n_cells for t in tabs], [t.r for t in tabs], [t.table_seed for t in tabs], opts)

        def call():
            return b.build_decode(dk, koff, out, koff, stream=stream)
        what = "pp_batch_build_decode, 4096 tables"
    else:
        n, r = cfg["n_cells"], cfg["r"]
        na, nb, nc = int(0.45 * n), int(0.30 * n), int(0.25 * n)
        keys = ppgen.distinct_keys(na + nb + nc, 31)
        dk = torch.from_numpy(keys.view(np.int64)).cuda()
        out = torch.empty(na + nb, dtype=torch.int64, device="cuda")
        sg = torch.empty(na + nb, dtype=torch.int8, device="cuda")
        t = pp.IBLT(n, r, 0x5195, opts)

        def call():
            t.build(dk[:nc + na], stream)
            t.delete(dk[:nc], stream)
            t.delete(dk[nc + na:], stream)
            return t.decode_signed(out, sg, stream=stream)
        what = f"build + pp_iblt_decode_signed, 2^{args.cells_log2} cells"
    for _ in range(2):
        call()
    torch.cuda.synchronize()
    ev[0].record(stream)
    call()
    ev[1].record(stream)
    stream.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "call": what, "ms": ev[0].elapsed_time(ev[1]),
                      "host_loop": bool(args.host_loop)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (4096 tables) and served (Poisson arrivals) sections")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="arrival window of the served section at the offered 20k req/s")
    ap.add_argument("--serve-below-seconds", type=float, default=10.0,
                    help="arrival window of the served section at 70 %% of the measured capacity")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive rounds from the host (kernels launched one by one, as profilers need)")
    ap.add_argument("--cells-log2", type=int, default=26,
                    help="table size for profiling runs (the benchmark itself is 2^26)")
    ap.add_argument("--profile-case", choices=["kcore", "plain", "batched", "signed", "served"],
                    help="for profilers: run one call of a secondary workload after two warm-up "
                         "calls, print its time and exit (no benchmark line)")
    ap.add_argument("--profile-c", type=float, default=0.70, help="density of --profile-case kcore")
    args = ap.parse_args()
    cfg = dict(ppgen.IBLT_HEADLINE)
    if args.cells_log2 != 26:
        cfg["n_cells"] = 1 << args.cells_log2
        cfg["name"] = f"iblt n=2^{args.cells_log2} r=3 c=0.75 (profiling size)"
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    import paper_1302_7014_b300 as pp

    if args.profile_case:
        profile_case(pp, torch, args, cfg)
        return

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, r, c = cfg["n_cells"], cfg["r"], cfg["c"]
    m = ppgen.edges_from_c(c, n)
    key_seed, table_seed = rank_workload(cfg, rank)
    keys_h = ppgen.distinct_keys(m, key_seed)
    stream = torch.cuda.Stream()
    table = pp.IBLT(n, r, table_seed, pp.options(host_loop=1) if args.host_loop else None)
    with torch.cuda.stream(stream):
        dkeys = torch.from_numpy(keys_h.view(np.int64)).cuda()
        out = torch.empty(m, dtype=torch.int64, device="cuda")
    stream.synchronize()

    def step(ev=None):
        # one pp_iblt_build_decode: the slab-binned build, whose tile write-out
        # also finds F_1, then the tile rounds
        if ev:
            ev[0].record(stream)
        res = table.build_decode(dkeys, out, stream=stream)
        if ev:
            ev[1].record(stream)
        return res

    def split_step(ev):
        # the same work as two calls (pp_iblt_build, then pp_iblt_decode, which
        # scans the table for F_1): the build / decode split of the step
        ev[0].record(stream)
        table.build(dkeys, stream)
        ev[1].record(stream)
        res = table.decode(out, stream=stream)
        ev[2].record(stream)
        return res

    clocks = ClockSampler(local)
    clocks.start()   # from before the warm-up: nvidia-smi takes a moment to start
    for _ in range(args.warmup):
        res = step()
    assert res.recovered == m and res.residual_cells == 0, "decode did not recover every key"
    rounds = res.rounds
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    recovered = 0
    for k in range(args.steps):
        res = step(evs[k])
        recovered += res.recovered
    t_end.record(stream)
    stream.synchronize()
    w1 = time.time()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop(w0, w1)
    total_ms = t_start.elapsed_time(t_end)
    fused_ms = [e[0].elapsed_time(e[1]) for e in evs]
    sevs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for k in range(args.steps):
        res = split_step(sevs[k])
        assert res.recovered == m and res.rounds == rounds
    stream.synchronize()
    build_ms = [e[0].elapsed_time(e[1]) for e in sevs]
    decode_ms = [e[1].elapsed_time(e[2]) for e in sevs]
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = sum_over_ranks(recovered, dist, "cuda") / (total_ms / 1000.0)

    # end to end through the public API: pinned host keys in, recovered keys out.
    # Every step copies its keys host -> device and its recovered keys back;
    # the copies run on their own streams, double-buffered, so step k's
    # download and step k+1's upload overlap step k's and k+1's compute (PCIe
    # is full duplex).
    e2e = None
    if not args.no_e2e:
        # through the library's host-buffer entry points: per step one
        # pp_iblt_submit_host (upload, build, decode and download enqueued by the
        # library, the copies on its own upload and download streams) and one
        # pp_iblt_finish_host; up to three steps in flight, so step k+1's upload
        # overlaps step k's decode and step k's download overlaps step k+1's
        # build and decode
        hk = torch.from_numpy(keys_h.view(np.int64)).pin_memory().numpy().view(np.uint64)
        outs = [torch.empty(m, dtype=torch.int64).pin_memory().numpy().view(np.uint64) for _ in range(3)]

        def pipeline(steps):
            got = 0
            tickets = [table.submit_host(hk, outs[k % 3], stream) for k in range(min(2, steps))]
            for k in range(steps):
                if k + 2 < steps:
                    tickets.append(table.submit_host(hk, outs[(k + 2) % 3], stream))
                res = table.finish_host(tickets[k])
                assert res.recovered == m
                got += res.recovered
            return got

        pipeline(2)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = pipeline(args.steps)
        torch.cuda.synchronize()
        e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, dist, "cuda")
        last = outs[(args.steps - 1) % 3]
        assert np.bitwise_xor.reduce(last) == np.bitwise_xor.reduce(keys_h) and last.sum() == keys_h.sum()
        e2e = {"value": sum_over_ranks(got, dist, "cuda") / (e_ms / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(m * 8), "d2h_bytes_per_step": int(m * 8),
               "ms_per_step": e_ms / args.steps, "api_calls_per_step": 2,
               "pipeline": "per step one pp_iblt_submit_host and one pp_iblt_finish_host (C ABI, pinned host "
                           "buffers, wall clock), three steps in flight; the library overlaps the uploads and "
                           "downloads of neighbouring steps with each step's build and decode"}
        # the floor the copies set: the same bytes up and down at once, pinned
        # memory, no kernels (PCIe and host memory are shared by both directions)
        d_up = torch.empty(m, dtype=torch.int64, device="cuda")
        d_dn = torch.zeros(m, dtype=torch.int64, device="cuda")
        hk_t = torch.from_numpy(hk.view(np.int64))
        ho_t = torch.from_numpy(outs[0].view(np.int64))
        cs = [torch.cuda.Stream(), torch.cuda.Stream()]
        ct = []
        for _ in range(4):
            torch.cuda.synchronize()
            c0 = time.perf_counter()
            with torch.cuda.stream(cs[0]):
                d_up.copy_(hk_t, non_blocking=True)
            with torch.cuda.stream(cs[1]):
                ho_t.copy_(d_dn, non_blocking=True)
            torch.cuda.synchronize()
            ct.append((time.perf_counter() - c0) * 1e3)
        c_ms = float(np.median(ct[1:]))
        e2e["copy_floor"] = {"ms": c_ms, "gb_s": 2 * m * 8 / (c_ms * 1e-3) / 1e9,
                             "frac": c_ms / e2e["ms_per_step"],
                             "what": "one step's upload and download at once (pinned, two streams, no kernels); "
                                     "frac = that time / the e2e step"}
        del outs, d_up, d_dn
        torch.cuda.empty_cache()

    # kernels of one step: k_bin, k_flag_to_host, k_ctl_init, n_slabs + 2
    # launches of the tile step for the 2^21-cell slabs (the build, finding
    # F_1 as it writes each tile out); the decode graph's k_trescan and
    # k_tprefix, six kernels per round (k_tclaim, k_tsort, k_tactive, k_tapply,
    # k_tapply_sparse, k_round_end) and k_trestore
    launches_per_step = 3 + (-(-n // (1 << 21)) + 2) + 2 + 6 * rounds + 1

    # roofline of the two halves of a step (sector-floor byte model)
    peak, peak_kind = hbm_peak()
    build_bytes = m * (8 + 64 * r)                 # key read + r cell sectors read+written
    # the scan's 4 B count per cell + per key r sector RMWs, the key out and its frontier entry
    decode_bytes = n * 4 + m * (64 * r + 16)
    # the fused step: the build's bytes and the decode's without its scan
    step_bytes = build_bytes + m * (64 * r + 16)
    b_ms, d_ms = float(np.mean(build_ms)), float(np.mean(decode_ms))
    s_ms = float(np.mean(fused_ms))
    kernels = {
        "step": {"kernel": "pp_iblt_build_decode: k_bin + k_tile_step per slab (the tile write-out also finds "
                           "F_1), then the decode graph (k_trescan, k_tprefix; per round k_tclaim, k_tsort, "
                           "k_tactive, k_tapply + k_tapply_sparse, k_round_end; k_trestore)",
                 "ms": s_ms, "bytes": step_bytes, "achieved_gbs": step_bytes / (s_ms * 1e-3) / 1e9,
                 "timed": "CUDA events around each pp_iblt_build_decode of the timed region"},
        "build": {"kernel": "k_bin + k_tile_step per slab (slab-binned, tiles in shared memory)", "ms": b_ms,
                  "bytes": build_bytes,
                  "achieved_gbs": build_bytes / (b_ms * 1e-3) / 1e9,
                  "timed": "pp_iblt_build alone, the same steps repeated after the timed region"},
        "decode": {"kernel": "decode graph (k_tscan, k_tprefix; per round k_tclaim, k_tsort, k_tactive, "
                             "k_tapply + k_tapply_sparse, k_round_end; k_trestore)", "ms": d_ms,
                   "bytes": decode_bytes, "achieved_gbs": decode_bytes / (d_ms * 1e-3) / 1e9,
                   "timed": "pp_iblt_decode alone (with its scan), after each pp_iblt_build above"},
    }
    for kk in kernels.values():
        kk["frac"] = kk["achieved_gbs"] / peak
    dom = "step"
    dk = kernels[dom]
    traffic = traffic_for(dom)
    roofline = {"bound": "hbm", "achieved": dk["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": dk["achieved_gbs"] / peak, "traffic": traffic,
                "kernel": dk["kernel"], "peak_source": f"{peak_kind} hbm_gbs",
                "model": "sector floor: (8+64r) B/key build + (64r+16) B/key rounds (the fused step reads "
                         "no cell for F_1); the split: 4 B/cell scan + (64r+16) B/key decode"}
    if traffic:
        # DRAM bytes the unit actually moves (ncu, committed summary) over the same time:
        # a random touch of a 32 B sector costs a 64 B read and its write-back, twice the model
        roofline["dram_gbs"] = traffic / (dk["ms"] * 1e-3) / 1e9
        roofline["dram_frac"] = roofline["dram_gbs"] / peak

    if world == 1 and not args.no_extra:
        # the same decode against what the GPU gives for its access pattern: per
        # recovered key r - 1 cells are read and written back, 2 (r - 1)
        # scattered 32 B accesses (the cell it was found in is emptied by the
        # write that made it pure, or by the streaming scan)
        sc = bench_scatter(pp, torch)
        rate = sc["tile_sorted_read_write"]["accesses_per_s"]
        per_key = 2 * (r - 1)
        ceiling = rate / per_key
        roofline["scatter_ceiling"] = {
            "accesses_per_s": rate, "accesses_per_key": per_key, "keys_per_s": ceiling,
            "decode_keys_per_s": m / (d_ms * 1e-3), "frac": m / (d_ms * 1e-3) / ceiling,
            "measured": sc}

    batched = served = subrounds = kcore = tables = signed = None
    if world == 1 and not args.no_extra:
        subrounds = bench_subrounds(pp, torch, table, dkeys, out, stream, m, max(3, min(args.steps, 5)))
        table.close()
        torch.cuda.empty_cache()
        del dkeys, out
        batched = bench_batched(pp, torch, args)
        torch.cuda.empty_cache()
        served = bench_served(pp, torch, args)
        torch.cuda.empty_cache()
        served["vs_plain_loop"] = bench_served_vs_plain(pp, torch, args)
        torch.cuda.empty_cache()
        kcore = bench_kcore(pp, torch, args)
        signed = bench_signed(pp, torch, args)
        tables = bench_tables(pp, torch, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(cfg)
        except Exception as exc:  # the baseline is informative only
            cpu = {"error": str(exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": cfg["name"], "n_cells": n, "r": r, "load": c, "keys": m,
                           "rounds": rounds, "l2": f"inputs > L2 ({n * 32 / 1e9:.2f} GB table, {m * 8 / 1e9:.2f} GB keys)",
                           "cell": "32 B: u64 key XOR, u64 checksum XOR, i32 count, padding",
                           "parallelism": f"replicas x{world}" if world > 1 else "single",
                           "round_loop": "host" if args.host_loop else "graph"},
                "build_ms": b_ms, "decode_ms": d_ms, "peel_ms": d_ms,
                "decode_keys_per_s": m / (d_ms * 1e-3),
                "kernels": kernels, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "batched": batched, "served": served, "subrounds": subrounds, "kcore": kcore,
                "paper_tables": tables, "signed": signed,
                "gpu_launches": args.steps * launches_per_step, "clocks": clk}
        print(json.dumps(line), flush=True)
    if batched is None:
        table.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
