"""CPU: the host logic of bench.py's multi-rank (replica) path, on two gloo
ranks: every timing is the maximum over the ranks, the job rate counts every
rank's units over the slowest rank's time, and the reference arm runs on
rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r times [1 + r, 10 - r, nan-free]: the maximum is taken per entry
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 5.0], world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 5.0]


def test_job_rate_and_single_rank():
    import bench
    assert bench.max_over_ranks([3.5, 1.0], 1) == [3.5, 1.0]  # no collective without a group
    # 2 ranks x 1e6 units, slowest rank 2 ms per step -> 1e9 units/s for the job
    assert bench.job_rate(2, 1e6, 2.0) == pytest.approx(1e9)


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of 2 exits 0 without work or output (rank 0 alone prints the line)
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_clock_summary_keeps_the_timed_window():
    # samples 20 ms apart: only those within the window (one interval of
    # slack) count; throttle reasons are those seen inside it
    import datetime
    import bench
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    lines = []
    for k in range(20):
        ts = t0 + datetime.timedelta(milliseconds=20 * k)
        sm = 2070 if 5 <= k <= 9 else 1200
        cap = "Active" if k == 15 else "Not Active"
        lines.append(f"{ts:%Y/%m/%d %H:%M:%S.%f}"[:-3] + f", 0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, "
                     f"Not Active, {cap}\n")
    got = bench.ClockSampler.summarize(lines, t0 + datetime.timedelta(milliseconds=110),
                                       t0 + datetime.timedelta(milliseconds=170))
    assert got["samples"] == 20 and got["samples_in_timed_region"] == 5
    assert got["sm_mhz"] == 2070 and got["reasons"] == []
    everything = bench.ClockSampler.summarize(lines)
    assert everything["samples_in_timed_region"] == 20 and everything["reasons"] == ["sw_power_cap"]
