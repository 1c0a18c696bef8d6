"""bench.py's multi-rank host logic on two gloo ranks (CPU): each rank owns
different rows, the job time is the slowest rank's, and the rate counts every
rank's rows."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    _, theta, _ = bench.rank_workload(rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    q.put((rank, float(theta[0, 0]), theta.shape[0], ms, bench.job_rate(theta.shape[0], world, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, b0, ms0, v0), (r1, t1, b1, ms1, v1) = res
    assert t0 != t1  # independent rows per rank
    assert ms0 == ms1 == 15.0  # the slowest rank's time on both ranks
    assert np.isclose(v0, 2 * b0 / 0.015) and v0 == v1


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_pool", lambda *a, **k: called.append(1))
    monkeypatch.setattr(bench, "oracle_rows_wall", lambda *a, **k: called.append(1) or 1.0)
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0
    assert not called and capsys.readouterr().out == ""


def test_reference_arm_reports_measured_step_time(monkeypatch, capsys):
    """ms_per_step is the wall time each step measured; value extrapolates the
    gradient's cost (central differences: 2 P + 1 evaluations per row)."""
    sys.path.insert(0, ROOT)
    import argparse
    import contextlib
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    walls = iter([9.0, 2.0, 4.0])  # one warm-up, two timed steps
    monkeypatch.setattr(bench, "oracle_pool", lambda *a, **k: contextlib.nullcontext())
    monkeypatch.setattr(bench, "oracle_rows_wall", lambda *a, **k: next(walls))
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 8)
    assert bench.run_reference(argparse.Namespace(gpus=1, steps=2, warmup=1)) == 0
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["ms_per_step"] == 3000.0
    rows = bench.REFERENCE_STEP_ROWS
    assert np.isclose(line["value"], rows / (3.0 * (2 * 20 + 1)))
    assert line["cpu_baseline"]["cores"] == rows and line["cpu_baseline"]["nproc"] == 8
