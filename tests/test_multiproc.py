"""The N > 1 path of bench.py on the CPU: gloo ranks and a torchrun launch.

Every GPU gets its own replica (its own table and keys: weak scaling, no
exchange on the data path); the job time is the slowest rank's and the job
throughput is the units of all ranks over that time.  These tests run the
host side of that with two gloo ranks, and the reference arm under torchrun
(rank 0 alone works and prints).
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import ppgen
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = dict(ppgen.IBLT_HEADLINE)
    assert bench.dist_setup() == (world, rank, rank)
    kseed, tseed = bench.rank_workload(cfg, rank)
    keys = torch.from_numpy(ppgen.distinct_keys(2000, kseed).view(np.int64))
    gathered = [torch.zeros_like(keys) for _ in range(world)]
    dist.all_gather(gathered, keys)
    seeds = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(seeds, torch.tensor([kseed, tseed], dtype=torch.int64))
    slow = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    units = bench.sum_over_ranks(1000 + rank, dist, "cpu")
    q.put((rank, [g.numpy() for g in gathered], [s.tolist() for s in seeds], slow, units))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, seeds, slow, units in out:
        # distinct replicas: other seeds, no shared key
        assert seeds[0] != seeds[1]
        assert np.intersect1d(gathered[0], gathered[1]).size == 0
        assert slow == 20.0 and units == 2001


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1     # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
