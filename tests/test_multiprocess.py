"""The multi-process path of the benchmark on CPU: world size 2 over gloo.

Runs are independent, so the benchmark shards nothing at run time: every rank
runs its own replica of the workload, and the only collectives are the timing
barrier and the max-over-ranks reduction of the elapsed time.  These tests run
those pieces (and the oracle arm under torchrun) on the host.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    r, w, dist = bench.dist_setup(world, backend="gloo")
    elapsed = 1.5 + r  # this rank's own time
    dist.barrier()
    worst = bench.max_over_ranks(elapsed, dist)
    value = bench.job_throughput(1000.0, w, worst)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, worst, value))


def test_barrier_and_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the job value counts both ranks' units
    assert out == [(0, 2, 2.5, 800.0), (1, 2, 2.5, 800.0)]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    env = dict(os.environ)
    os.environ.pop("RANK", None)
    try:
        assert bench.dist_setup(1) == (0, 1, None)
        assert bench.max_over_ranks(3.0, None) == 3.0
        assert bench.job_throughput(10.0, 1, 2.0) == 5.0
    finally:
        os.environ.clear()
        os.environ.update(env)


def test_oracle_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched like the GPU arm (torchrun, 2
    processes): rank 0 alone times the oracle and prints one JSON line; the other
    rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
