"""The N > 1 path on CPU ranks (gloo, world size 2).

The batched workloads shard as replicas: every rank solves its own copy of
the batch, there is no data-path collective, and the job's time is the
slowest rank's.  These tests run that host logic (process-group setup from
the torchrun environment, max over ranks, whole-job rate, rank-0-only
output of the reference arm) as real processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    r, w, local = bench._dist("gloo")
    try:
        # the slowest rank's time bounds the job
        ms = bench.rank_max(10.0 + 5.0 * r, w, device="cpu")
        rate = bench.job_rate(1000, w, ms)
        dist.barrier()
        out.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_rank_max_and_job_rate_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, w, local, ms, rate in res:
        assert w == world and local == r
        assert ms == 15.0                      # max over ranks, on every rank
        assert rate == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_needs_no_process_group():
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK")}
    saved = dict(os.environ)
    try:
        os.environ.clear()
        os.environ.update(env)
        assert bench._dist("gloo") == (0, 1, 0)
        assert bench.rank_max(3.5, 1) == 3.5
        assert bench.job_rate(262144, 1, 2.0) == pytest.approx(262144 / 0.002)
    finally:
        os.environ.clear()
        os.environ.update(saved)


def test_reference_arm_under_torchrun_prints_once():
    """Under torchrun only rank 0 runs the oracle arm and prints its line;
    the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="4")
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(x) for x in res.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["metric"] == bench.METRIC and line["unit"] == "stage-solves/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["value"] > 0
