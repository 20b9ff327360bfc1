"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the job
time is the slowest rank's, the rate counts every replica's steps, and under
--impl reference only rank 0 prints."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms = 100.0 + 50.0 * rank                  # rank 1 is the slow one
    got = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.job_rate(10, world, got)
    out.put((rank, got, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == 150.0
        assert abs(rate - 2 * 10 / 0.15) < 1e-9


def test_reference_arm_prints_on_rank0_only():
    """Under torchrun the reference arm's non-zero ranks exit 0 silently."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0",
                        "--workload", "d2_D2_chi16"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert abs(bench.job_rate(200, 1, 1000.0) - 200.0) < 1e-12
