"""Host logic of the multi-rank bench (replicas, one per GPU): the whole-job
time is the slowest rank's, pairs add up over ranks, throughput counts every
rank's particles.  Runs as two gloo ranks on the CPU; the reference arm of a
non-zero rank exits without work."""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.0, 20.0][rank]
        pairs = [1000.0, 3000.0][rank]
        max_ms, total_pairs = bench.reduce_over_ranks(ms, pairs, dist, device="cpu")
        value = bench.job_throughput(4000, 10, world, max_ms)
        out.put((rank, max_ms, total_pairs, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, total_pairs, value in results:
        assert max_ms == 20.0 and total_pairs == 4000.0
        assert value == pytest.approx(4000 * 10 * 2 / 0.020)


def test_reference_arm_on_a_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
