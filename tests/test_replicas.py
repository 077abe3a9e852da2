"""Multi-GPU path on the CPU: bench.py runs independent replicas (the right-hand
sides and problems of this workload need no exchange between GPUs), reports
the job time as the slowest replica's and the whole-job rate over all ranks.
Here two gloo ranks exercise that host logic; no GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, elapsed, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(elapsed[rank], dist, "cpu")
        out.put((rank, t, bench.replica_rate(world, 64, 2, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_replica():
    world, elapsed = 2, [3.0, 5.0]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, elapsed, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(world))
    for rank, t, rate in got:
        assert t == 5.0                              # every rank sees the slowest time
        assert rate == pytest.approx(2 * 64 * 2 / 5.0)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.replica_rate(1, 64, 1, 2.0) == 32.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle; the others exit at once."""
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "cpu_sample", lambda *a, **k: called.append(a) or (1.0, 1, 1.0))

    class Args:
        n, warmup, steps, gpus = 31, 3, 1, 2
        schedule, b_aux = bench.DEFAULT_SCHEDULE, bench.DEFAULT_B_AUX
    bench.run_reference(Args())
    assert called == [] and capsys.readouterr().out == ""
    # rank 0 prints one line on the GPU arm's metric and unit, with its cores stated
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(Args())
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "RHS-solves/s" and line["metric"] == bench.METRIC
    assert line["cpu_baseline"]["cores"] == 1 and len(called) == Args.warmup + Args.steps
    assert line["config"]["schedule"] == Args.schedule and line["config"]["b_aux"] == Args.b_aux
