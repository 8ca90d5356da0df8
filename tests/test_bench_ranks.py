"""The replica path of bench.py on CPU: two gloo ranks.

Multi-GPU runs of the filter are replicas (nothing is sharded, no data-path
collective); what crosses ranks is the max over ranks of the timed region and
the whole-job rate, which counts every replica's cell-steps over the slowest
replica's time.  Under torchrun the reference arm runs on rank 0 only; the
other ranks exit 0 without work.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(times[rank], world, "cpu")
        out.put((rank, slowest, bench.whole_job_rate(world, 1e9, slowest)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(1500.0, 2000.0), (3000.0, 250.0)])
def test_two_replicas_report_the_slowest_rank(times):
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    for rank, got, rate in res:
        assert got == slowest, (rank, got)
        # 2 ranks x 1e9 cell-steps over the slowest rank's seconds, in G
        assert rate == pytest.approx(2 * 1e9 / (slowest / 1e3) / 1e9, rel=1e-15)


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(1, 6.0e9, 1000.0) == pytest.approx(6.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
