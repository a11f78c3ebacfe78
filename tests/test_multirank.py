"""Host logic of the multi-rank benchmark (replicas: one independent solve per
rank, no data-path collective) on CPU with gloo, world size 2."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    slow = bench.max_over_ranks(1.0 + rank)             # rank 1 is the slowest
    rate = bench.aggregate_rate(1000.0, 2.0 + 3.0 * rank, ws)
    q.put((r, ws, local, slow, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, local, slow, rate) in enumerate(out):
        assert (rank, ws, local) == (r, 2, r)
        assert slow == 2.0
        assert rate == pytest.approx(1000.0 * 2 / 5.0)   # units of both ranks / slowest time


def test_reference_arm_runs_on_rank0_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"config": "flat2d", "steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.reference_arm(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_json_line(capsys, monkeypatch):
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), {"config": "flat2d", "steps": 2, "warmup": 1, "gpus": 1})()
    assert bench.reference_arm(args) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
