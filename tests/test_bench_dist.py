"""Multi-process logic of the benchmark on CPU (gloo, world size 2).

Under torchrun every rank back-projects its own replica of the workload;
the only cross-rank steps are the barrier and the max-over-ranks of the
timed region, and the value is the updates of all replicas over the slowest
replica's time.  The reference arm (the oracle on host cores) runs on rank 0
alone.  These tests run those steps as two gloo processes on the CPU.
"""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist()
        # each replica "took" a different time; the job takes the slowest
        ms = bench._max_over_ranks(10.0 + 5.0 * rank, w, torch.device("cpu"))
        rate = bench._job_rate(w, 6.0e10, ms * 1e-3)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"world": w, "rank": r, "local": local, "ms": ms, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, g in enumerate(got):
        assert (g["world"], g["rank"], g["local"]) == (world, r, r)
        assert g["ms"] == 15.0                       # max over ranks, seen by every rank
        assert g["rate"] == pytest.approx(2 * 6.0e10 / 15e-3 / 1e9)


def test_single_process_needs_no_group():
    import bench
    assert bench._max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench._job_rate(1, 1e9, 1.0) == 1.0


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    """A non-zero rank of the reference arm exits 0 at once: it neither
    builds nor runs the oracle and prints nothing."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    import oracle

    def boom(*a, **k):
        raise AssertionError("rank 1 must not touch the oracle")

    monkeypatch.setattr(oracle, "build", boom)
    monkeypatch.setattr(oracle, "backproject", boom)
    args = type("A", (), {"config": "fdk512", "steps": 1, "warmup": 0, "gpus": 2,
                          "ref_step_seconds": 1.0})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank0(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle on a bounded slab of the
    named workload and prints one JSON line with the bench contract's keys
    (here on the small test scan, so it runs in a second on the CPU)."""
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = type("A", (), {"config": "small", "steps": 2, "warmup": 1, "gpus": 1,
                          "ref_step_seconds": 0.05, "proj_dtype": "f32"})()
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GUp/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 1)
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert line["config"]["workload"].startswith("small: 24x20x18")
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"] and cpu["cores"] >= 1
    assert "slab" in cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "GUp/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
