"""The multi-GPU path of bench.py is replicas (one independent search per
rank, no data-path collective): the job's time is the slowest rank's and
its rate counts every rank's curves.  Checked here with two gloo ranks on
the CPU, including the reference arm's rank-0-only rule."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, times, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    dist.barrier()
    t = bench.max_over_ranks(times[rank])
    q.put((rank, t, bench.job_rate(world, 5, t)))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [3.0, 4.5]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [4.5, 4.5]
    # 2 ranks x 5 curves in 4.5 s
    assert out[0][2] == pytest.approx(2 * 5 * 3600.0 / 4.5)


def test_single_process_is_not_distributed():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_rate(1, 4, 2.0) == pytest.approx(7200.0)


def test_reference_arm_runs_on_rank_zero_only():
    # a non-zero rank of the reference arm exits 0 without work or output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
