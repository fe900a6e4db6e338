"""The benchmark's multi-rank harness on CPU: two gloo ranks on 127.0.0.1.

With N ranks every rank runs an independent replica; the timed region is
bracketed by barriers, the step time is the maximum over ranks, the value is
N times one replica's edges over that time, and only rank 0 prints. The
reference arm under N ranks runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r = bench.Replicas("gloo", "cpu")
    assert (r.rank, r.world) == (rank, world)
    r.barrier()
    step_s = 0.002 * (rank + 1)  # rank 1 is the slower replica
    slowest = r.max(step_s)
    value = r.aggregate_gteps(1_000_000, slowest)
    r.barrier()
    r.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "value": value}, f)


def test_two_gloo_ranks_take_the_slowest_step(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == pytest.approx(0.004)
        # 2 replicas x 1e6 edges in 4 ms = 0.5 GTEPS
        assert r["value"] == pytest.approx(0.5)


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    r = bench.Replicas("gloo", "cpu")
    assert r.world == 1 and r.dist is None
    r.barrier()
    assert r.max(0.25) == 0.25
    assert r.aggregate_gteps(3_000_000, 0.001) == pytest.approx(3.0)
    r.close()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    assert bench.run_reference(bench.parse_args()) == 0
    assert capsys.readouterr().out == ""
