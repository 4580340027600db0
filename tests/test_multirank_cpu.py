"""The N > 1 paths on the CPU with gloo ranks (no GPU).

The samples of one update are independent, so Eq. 4 shards over devices by
splitting K: each shard reduces to (m_g, Z_g, N_g) and a log-sum-exp merge
gives the full update.  These tests run that exchange among two gloo ranks
with the oracle, and the benchmark's own multi-rank logic (slowest-rank
timing; one JSON line from rank 0) under torchrun.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2609_02020_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def case():
    arm = synth.arm(3)
    q, qd = synth.state(1003, arm)
    return dict(rb=oracle.make_robot(arm), oc=oracle.make_cost(synth.cost_free_space()),
                q=q, qd=qd, goal=synth.goal(1003, arm), T=6, K=64, lam=1.0)


def shard(c, k0, k1):
    S, noise = [], []
    for k in range(k0, k1):
        s, nz = oracle.rollout(c["rb"], c["oc"], 0.01, c["T"], np.full(7, 2.0), 9, 0, k, c["q"],
                               c["qd"], c["goal"], synth.NO_PLANE, np.zeros((c["T"], 7)),
                               want_noise=True)
        S.append(s)
        noise.append(nz)
    return np.array(S), np.array(noise)


def test_partial_merge_equals_full_update_for_any_split():
    rng = np.random.default_rng(0)
    K, T, n = 40, 5, 7
    S = rng.uniform(0, 30, K)
    S[7] = np.nan
    noise = rng.normal(size=(K, T, n))
    plan = rng.normal(size=(T, n))
    _, full, full_next, _ = oracle.mppi_update(S, noise, plan, 0.7)
    for cuts in ([20], [1, 39], [5, 6, 30], [0, 40]):
        edges = [0] + cuts + [K]
        parts = [oracle.mppi_partial(S[a:b], noise[a:b].reshape(b - a, T, n) if b > a
                                     else np.zeros((0, T, n)), 0.7)
                 for a, b in zip(edges[:-1], edges[1:])]
        rc, us, nxt = oracle.mppi_merge(np.array(parts), plan, 0.7)
        assert rc == 0
        assert np.allclose(us, full, atol=1e-13) and np.allclose(nxt, full_next, atol=1e-13)


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = case()
        per = c["K"] // world
        S, noise = shard(c, rank * per, (rank + 1) * per)
        part = torch.tensor(oracle.mppi_partial(S, noise, c["lam"]))
        parts = [torch.zeros_like(part) for _ in range(world)]
        dist.all_gather(parts, part)
        rc, us, _ = oracle.mppi_merge(torch.stack(parts).numpy(), np.zeros((c["T"], 7)), c["lam"])
        import bench
        mx = bench.max_over_ranks([float(rank + 1), 10.0 - rank], world, "cpu")
        q.put((rank, rc, us, mx))
    finally:
        dist.destroy_process_group()


def test_sharded_update_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    sys.path.insert(0, ROOT)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    c = case()
    S, noise = shard(c, 0, c["K"])
    _, full, _, _ = oracle.mppi_update(S, noise, np.zeros((c["T"], 7)), c["lam"])
    for rank, rc, us, mx in res:
        assert rc == 0
        assert np.allclose(us, full, atol=1e-12)
        assert mx == [2.0, 10.0]


def test_bench_reference_arm_under_torchrun_prints_once():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1",
           "--K", "256", "--budget-s", "3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
