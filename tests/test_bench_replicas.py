"""The N-replica path of bench.py on CPU: two gloo ranks check the barrier,
the max-over-ranks timing and the whole-job rate, and that the reference arm
does its work on rank 0 only.  (bench.py on N GPUs runs N independent
replicas of the workload; there is no data-path collective to test.)"""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench._barrier(world)
        slowest = bench._max_over_ranks(world, 10.0 + rank)  # rank 1 is slower
        q.put((rank, slowest, bench.whole_job_rate(world, 1e9, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in res:
        assert slowest == 11.0
        # 2 ranks x 1e9 point-steps in 11 ms
        assert rate == pytest.approx(2 * 1e9 / 11e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's rank 1 exits 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_rate_is_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1, 6.7e10, 1000.0) == pytest.approx(67.0)
    assert bench.whole_job_rate(4, 6.7e10, 1000.0) == pytest.approx(4 * 67.0)


def test_reference_arm_times_a_variant_workload():
    """--impl reference --workload heat512: the oracle on that workload, one JSON line."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "heat512", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert "512" in line["config"]["reference_sample"]
