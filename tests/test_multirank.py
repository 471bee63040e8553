"""The replicas-only multi-GPU path of bench.py, on two gloo ranks (CPU):
each rank gets its own seeds, the job time is the slowest rank's, and the
whole-job rate counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, _ = bench.main_workload("ising1024", rank, 0)
        gathered = [None] * world
        dist.all_gather_object(gathered, list(w.seeds))
        slowest = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        rate = bench.whole_job_rate(w.steps_per_schedule() * w.schedules, 3, world, slowest)
        out[rank] = {"seeds": gathered, "slowest": slowest, "rate": rate,
                     "units": w.steps_per_schedule() * w.schedules}
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_replicas_and_take_slowest_time():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    r0, r1 = out[0], out[1]
    # every rank sees the same gathered seed lists, and the ranks' replicas differ
    assert r0["seeds"] == r1["seeds"]
    assert not set(r0["seeds"][0]) & set(r0["seeds"][1])
    # the job's time is the slowest rank's; the rate counts both ranks' units
    assert r0["slowest"] == r1["slowest"] == 2.0
    assert r0["rate"] == r0["units"] * 3 * world / 2.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, schedules, warmup, steps, gpus = "ising1024", 0, 0, 1, 2
    assert bench.reference_arm(A()) == 0  # returns at once, no oracle work


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle and prints one JSON line
    with the benchmark contract's keys (the arms' ratio is computed from it)."""
    import json
    import bench
    monkeypatch.setenv("RANK", "0")

    class A:
        workload, schedules, warmup, steps, gpus = "ising1024", 0, 0, 1, 1
    assert bench.reference_arm(A()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["config"]["workload"].startswith("1024x1024")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
