"""The bench's N > 1 path on CPU: two gloo ranks (the GPU runs use one NCCL rank per GPU).

Every rank renders its own replica of the workload, so the only cross-rank steps are the timing
reduction (the job's time is its slowest rank's) and rank 0's report; the reference arm runs on
rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        slowest = bench.max_over_ranks(seconds[rank], w, torch.device("cpu"))
        q.put((r, w, local, slowest, bench.job_rate(w, 10, slowest)))
    finally:
        dist.destroy_process_group()


def test_timing_reduction_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    seconds = [1.25, 2.5]  # rank 1 is the slower one
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, slowest, rate) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == max(seconds)  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 10 / max(seconds))  # all ranks' iterations over that time


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_env() == (1, 0, 0)
        assert bench.max_over_ranks(3.0, 1, None) == 3.0
        assert bench.job_rate(1, 200, 0.5) == 400.0
    finally:
        os.environ.update(saved)
