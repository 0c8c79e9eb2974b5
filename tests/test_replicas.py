"""The N>1 bench path on CPU: two `gloo` ranks, each a replica of the whole
workload (the path has no exchange step, so no collective touches the data).
Checks the timing reduction (max over ranks), the whole-job throughput and
that only rank 0 runs and prints the reference arm."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # each replica times its own steps; the slowest one sets the job's time
        local_ms = 10.0 + 7.5 * rank
        job_ms = bench.max_over_ranks(local_ms, dist)
        units, steps = 2 * 2048 * 2048, 5
        value = bench.job_throughput(world, units, steps, job_ms * 1e-3)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"local_ms": local_ms, "job_ms": job_ms, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    slowest = max(r["local_ms"] for r in res)
    for r in res:
        assert r["job_ms"] == slowest
        # every rank reports the same whole-job number: all units over the slowest time
        assert r["value"] == pytest.approx(world * 2 * 2048 * 2048 * 5 / (slowest * 1e-3), rel=1e-12)


def test_single_process_is_identity():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_throughput(1, 100, 4, 2.0) == 200.0


def test_reference_arm_other_ranks_idle(monkeypatch, capsys):
    class Args:
        gpus, steps, warmup = 2, 1, 3

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(monkeypatch, capsys):
    """`bench.py --impl reference` on rank 0: one JSON line with the contract's
    keys, the oracle as the timed program (a tiny bounded sample here)."""
    class Args:
        gpus, steps, warmup = 1, 1, 3

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("SDF_REF_NODES", "512")
    assert bench.run_reference(Args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == bench.WORKLOAD
