"""Host logic of bench.py on the CPU: the N > 1 path (replicas, whole-job throughput over the slowest rank)
with two gloo ranks, and the reference arm, which prints one JSON line on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [10.0, 20.0][rank]  # rank 1 is the slow one
        rate, slowest = bench.whole_job_rate(torch, dist, local_ms, 100.0, "cpu")
        out.put((rank, rate, slowest))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest time (20 ms) and the units of both ranks: 2 x 100 / 0.020 s
    for rank, rate, slowest in res:
        assert slowest == 20.0
        assert rate == pytest.approx(10000.0)


def test_single_process_rate():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    rate, slowest = bench.whole_job_rate(torch, None, 4.0, 8.0, "cpu")
    assert slowest == 4.0 and rate == pytest.approx(2000.0)


def run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(world),
                           "--steps", "1", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_prints_on_rank_0_only():
    r1 = run_reference(1, 2)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = run_reference(0, 2)
    assert r0.returncode == 0
    lines = [l for l in r0.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "config", "cpu_baseline",
                "e2e"):
        assert key in d
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_pool_reproduces_the_oracle_action():
    """The host-parallel timing harness of the oracle (bench.OraclePool) adds up exactly what the oracle's
    own Problem.apply computes, on the same problem, over the whole mesh and over a leading sample of cells."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from paper_1904_13131_gb300 import inputs
    m = 4
    pool = bench.OraclePool(m, workers=3)
    try:
        x = inputs.gaussian_vector(pool.n, seed=1)
        u = inputs.smooth_field(bench.DIM, bench.K, m, seed=0)
        ref = pool.P.apply(u, x)
        np.testing.assert_allclose(pool.apply(x), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        part = np.zeros(pool.n)
        xin = np.where(pool.P.constrained, 0.0, x)
        pool.P.apply_cells(u, xin, np.arange(40), part)
        np.testing.assert_allclose(pool.apply(x, 40), part, rtol=0, atol=1e-13 * np.abs(part).max())
    finally:
        pool.close()
