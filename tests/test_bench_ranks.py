"""The multi-rank arithmetic of bench.py (N independent replicas on N
GPUs, weak scaling): two gloo processes on CPU with unequal times agree on
the slowest rank's time and the whole-job rate; the reference arm runs on
rank 0 only."""
import importlib.util
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = load_bench()
    ms = [10.0, 12.5][rank]
    slow = b.slowest_over_ranks(ms, world)
    rate = b.job_rate(world, 1000.0, slow / 1e3)
    dist.barrier()
    q.put((rank, slow, rate))
    dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [12.5, 12.5]
    assert all(abs(o[2] - 2 * 1000.0 / 0.0125) < 1e-6 for o in out)


def test_single_rank_is_identity():
    b = load_bench()
    assert b.slowest_over_ranks(7.0, 1) == 7.0
    assert b.job_rate(1, 50.0, 2.0) == 25.0


def test_reference_arm_only_on_rank_zero():
    """under torchrun the reference arm prints on rank 0 only; the other
    ranks exit 0 without work"""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
