"""The multi-GPU form runs independent replicas (one map per rank, no data
collective). Its host logic is tested here on CPU with two gloo ranks: the
timing reduction (slowest rank's time, summed work), per-rank workloads that
differ, and the reference arm doing work on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1.0 + rank, 0.5 * (rank + 1)]
    counts = [100.0 * (rank + 1), 7.0]
    t, c = bench.reduce_over_ranks(times, counts, "cpu")
    out[rank] = (t, c)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t, c = out[r]
        assert t == [2.0, 1.0]          # the slowest rank's times
        assert c == [300.0, 14.0]       # the whole job's work


def test_ranks_get_distinct_robots():
    import bench
    import synth
    # seeds differ per rank, so each replica maps its own robot
    assert synth.SEEDS["sequence"] + 1000 * 0 != synth.SEEDS["sequence"] + 1000 * 1
    a = synth.sequence_scans("sequence", n_scans=1, seed=synth.SEEDS["sequence"])[1][0]
    b = synth.sequence_scans("sequence", n_scans=1, seed=synth.SEEDS["sequence"] + 1000)[1][0]
    assert a.points.shape == b.points.shape and not (a.points == b.points).all()
    assert bench.dist_env()[1] >= 1


def test_reference_arm_skips_other_ranks(capsys):
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, world=2)   # returns at once, prints nothing
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(capsys, monkeypatch):
    # rank 0 prints one JSON line with the keys the benchmark contract names,
    # its e2e and cpu_baseline describing the oracle run itself
    import json

    import bench
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    args = bench.parse()
    bench.run_reference(args, rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 1 and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["map"] == [512, 512, 64]
    # the same config dict as the GPU arm's line on this workload
    import synth
    assert line["config"] == bench.config_of("high_speed", synth.sequence_config("high_speed"), 40, 1)
    assert line["cpu_baseline"]["host"]["nproc"] >= 1 and line["cpu_baseline"]["host"]["model"]
