"""The multi-GPU path of the benchmark is N independent replicas (one update of one
reconstruction is one GPU's work): the host logic that joins them, run here as two gloo
ranks on the CPU.  Each rank reports its own timed milliseconds; every rank must get the
slowest one, and the whole-job value is the updates of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_of_rank, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        ms, value = bench.combine_ranks(ms_of_rank[rank], 10, world)
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ms_of_rank = [750.0, 800.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms_of_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in got:
        assert ms == 800.0
        assert value == pytest.approx(2 * 10 / 0.8)


def test_one_rank_is_its_own_time():
    import bench
    assert bench.combine_ranks(500.0, 10, 1) == (500.0, 20.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; the other ranks exit quietly."""
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0, cpu_fans=2, prec="bf16x3")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 times the oracle on a bounded sample and prints one line in the bench's
    format: the same metric, unit and config as the GPU arm, a cpu_baseline that
    describes the run (each step a fixed fraction of an update, fans and pixels alike),
    and an e2e object with no host-device traffic."""
    import argparse
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, cpu_fans=2, prec="bf16x3"))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    frac = 2 / 256
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * frac / d["value"]) < 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "2/256 fans" in cb["sample"]
    assert cb["update_fraction_per_step"] == frac and "2048/262144 pixels" in cb["sample"]
    assert d["config"] == bench.workload_config(bench.WORKLOAD, "bf16x3", 1)
    assert d["e2e"] == {"value": d["value"], "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD
