"""The multi-rank host logic of bench.py on CPU: world-size-2 gloo process groups.

The step does not shard (every box has one GPU, and one view's step needs no
exchange), so `bench.py --gpus N` runs N independent replicas under torchrun. What
the ranks share is the timing: a barrier on both sides of the timed region, the
slowest rank's time, and the whole-job rate over it. The reference arm runs on rank
0 only; the other ranks exit without work.
"""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(times[rank])
        rate = bench.job_rate(10, world, slowest)
        dist.barrier()
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate_over_two_gloo_ranks():
    times = [0.25, 0.4]  # seconds each rank took for its 10 steps
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == 0.4  # every rank sees the slowest replica's time
        assert abs(rate - 2 * 10 / 0.4) < 1e-9  # units of both ranks over that time


def test_without_a_process_group_the_values_are_the_rank_own():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.job_rate(20, 1, 0.5) == 40.0


def test_reference_arm_on_a_second_rank_exits_without_output():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
