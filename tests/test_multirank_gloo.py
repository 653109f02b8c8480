"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2).

With N GPUs each rank advances its own ensemble member (no collective on the data path); the
only collectives are the barrier and the max over ranks of the timed region.  These tests run
that logic in two processes over gloo, and check that the reference arm, which is the host-side
oracle, runs on rank 0 alone.
"""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    ms_max = bench.slowest(local_ms, dist, "cpu")
    dist.barrier()
    value = bench.job_throughput(world, 1024, 100, ms_max * 1e-3)
    q.put((rank, ms_max, value, bench.ensemble_seed(rank)))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    # every rank sees the slowest rank's time; the value counts both ranks' work
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 1024 * 100 / 0.015)
    # distinct ensemble members
    assert res[0][3] != res[1][3]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line(tmp_path):
    """Rank 0 of the reference arm prints one JSON line with the oracle's throughput."""
    import json

    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "particle-steps/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_launch_count_of_the_step_graph():
    import bench

    # commit + predictor + branch condition + (filter | five re-sort kernels) + passes B, C, D
    assert bench.launches_in_steps(1, 0) == 7
    assert bench.launches_in_steps(1, 1) == 11
    assert bench.launches_in_steps(100, 7) == 728
    assert set(bench.RESORT_BRANCH) | {"predict", "pass_a", "pass_b", "pass_c", "pass_d"} == set(
        bench.FLOPS_PER_PAIR) | {"predict", "cell_keys", "cell_scan", "cell_scatter", "cell_order"}
