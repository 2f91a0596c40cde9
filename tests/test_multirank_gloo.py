"""Multi-rank host logic on CPU (gloo, world size 2).

On one box the path runs as independent replicas; across GPUs the natural
exchange is one scalar per rank.  These tests cover that exchange's
arithmetic with CPU ranks reducing shards with the oracle, the max-over-ranks
timing rule of bench.py, and bench.py's reference arm under torchrun."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 1 << 20
    xf = workloads.uniform_f32(n, seed=0)
    xi = workloads.uniform_i32(n, seed=0)
    lo, hi = rank * n // world, (rank + 1) * n // world
    # each rank reduces its shard; the exchange is one scalar per rank
    sf = torch.tensor([oracle.sum_f32(xf[lo:hi])], dtype=torch.float64)
    si = torch.tensor([oracle.sum_i32(xi[lo:hi])], dtype=torch.int64)
    dist.all_reduce(sf, op=dist.ReduceOp.SUM)
    dist.all_reduce(si, op=dist.ReduceOp.SUM)
    # max-over-ranks timing: the slowest rank defines the step time
    t = torch.tensor([1.0 + rank * 0.25], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    if rank == 0:
        q.put((float(sf.item()), int(si.item()), float(t.item())))
    dist.destroy_process_group()


def test_shard_and_scalar_exchange_gloo():
    import oracle
    import workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sf, si, tmax = res
    n = 1 << 20
    xf = workloads.uniform_f32(n, seed=0)
    xi = workloads.uniform_i32(n, seed=0)
    assert si == oracle.sum_i32(xi)                       # integers: exact after the exchange
    exact = oracle.to_float(oracle.exact_f32(xf))
    assert abs(sf - exact) <= (n + 2) * 2.0 ** -53 * oracle.sum_abs_f32(xf)
    assert tmax == 1.25


def test_bench_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                               # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
