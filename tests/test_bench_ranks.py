"""bench.py's multi-rank bookkeeping (replicas: every rank runs the whole pass
on its own X) under two gloo ranks on the CPU: the job's time is the slowest
rank's, the value counts every rank's bytes, and only rank 0 runs the
reference arm."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 0.5 + rank  # rank 1 is the slow one
    t_max = bench.time_over_ranks(t_local, world)
    gbs = bench.job_gbs(2e9, 10, world, t_max)
    dist.destroy_process_group()
    q.put((rank, t_max, gbs))


def test_time_is_max_over_ranks_and_value_counts_all_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in res] == [1.5, 1.5]
    assert all(g == pytest.approx(2e9 * 10 * 2 / 1.5 / 1e9) for _, _, g in res)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.time_over_ranks(0.25, 1) == 0.25
    assert bench.job_gbs(4e9, 5, 1, 2.0) == pytest.approx(10.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-rows", "1000"], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_reference_arm_line_contract():
    # rank 0 prints one JSON line with the reference arm's keys: the oracle on
    # a bounded sample of the same workload, no host-device traffic
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-rows", "2000"], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    b = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert b["impl"] == "reference" and b["metric"] == bench.METRIC and b["unit"] == "GB/s"
    assert b["value"] > 0 and b["higher_is_better"] is True and b["steps"] == 1
    assert b["cpu_baseline"]["kind"] == "oracle" and b["cpu_baseline"]["cores"] >= 1
    assert b["cpu_baseline"]["value"] == b["value"]
    assert b["e2e"] == {"value": b["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert b["config"]["workload"] and b["config"]["parallelism"] == "single GPU"
