"""The replicas-only multi-GPU path of the benchmark, on CPU with the gloo
backend and two ranks: the barrier, the max over ranks of the timings, the
whole-job aggregate, and a reference arm that only rank 0 prints."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    class A:
        pass
    w, r, _ = bench.dist_setup(A())
    bench.barrier(w)
    slowest = bench.max_over_ranks(w, 10.0 + rank, "cpu")
    q.put((r, w, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    assert out == [(0, 2, 11.0), (1, 2, 11.0)]


def test_job_throughput_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.job_throughput(1, 1000, 8, 2.0)
    assert bench.job_throughput(2, 1000, 8, 2.0) == pytest.approx(2 * one)
    assert one == pytest.approx(1000 * 8 / 2e-3 / 1e6)


def test_reference_arm_under_two_ranks_prints_once():
    """torchrun with two ranks on 127.0.0.1: rank 0 times the oracle on a
    tiny sample and prints one JSON line; rank 1 exits without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
