"""The N > 1 path of the benchmark (independent replicas) with the gloo
backend on CPU: rank bookkeeping, barrier, max-over-ranks timing and the
whole-job throughput; and the CPU reference arm's rank gating."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    from paper_2503_22227_gb300 import replicas
    r, w, local = replicas.init_from_env("gloo")
    replicas.barrier(w)
    elapsed = 1.0 + r                      # rank 1 is the slowest
    slowest = replicas.max_over_ranks(elapsed, w, device="cpu")
    q.put((r, w, local, slowest, replicas.throughput(8 * 100, w, slowest)))
    replicas.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replicas_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1]
    for r, w, local, slowest, value in got:
        assert w == 2 and local == r
        assert slowest == 2.0
        assert value == pytest.approx(2 * 800 / 2.0)


def test_single_process_needs_no_group():
    from paper_2503_22227_gb300 import replicas
    env = {k: os.environ[k] for k in ("RANK", "WORLD_SIZE") if k in os.environ}
    try:
        for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
            os.environ.pop(k, None)
        assert replicas.init_from_env() == (0, 1, 0)
        assert replicas.max_over_ranks(3.5, 1) == 3.5
        assert replicas.throughput(10, 1, 2.0) == 5.0
    finally:
        os.environ.update(env)


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "3"],
                         env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""
