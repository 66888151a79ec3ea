"""The multi-rank side of bench.py on the CPU: two gloo ranks, as torchrun
would start them on two GPUs (replicas: no data-path collective; the timing
is the slowest rank's, the value the whole job's)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = [3.0, 7.5][rank]                       # this rank's timed region (s)
        t_max = bench.reduce_max(t, world, "cpu")
        rate = bench.whole_job_rate(1000.0, world, t_max)
        dist.barrier()
        q.put((rank, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_the_whole_job_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, rate in got:
        assert t_max == 7.5                      # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 7.5)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(4.25, 1) == 4.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the reference arm runs on rank 0 alone; another rank
    exits 0 at once without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=120, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    """Rank 0 of the reference arm times the CPU oracle on its bounded sample
    and prints one line with the contract's keys."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0", ORACLE_THREADS="4")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 4
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["metric"] == "relaxations/s (n^3/t)" and d["higher_is_better"] is True


def test_step_stats():
    sys.path.insert(0, ROOT)
    import bench
    s = bench.step_stats([3.0, 1.0, 2.0, 10.0])
    assert s == {"mean": 4.0, "median": 2.5, "min": 1.0, "max": 10.0, "n": 4}
