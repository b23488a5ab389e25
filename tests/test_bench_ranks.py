"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): the step
time is the slowest rank's, the whole-job value divides it by N, and the
reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = 10.0 + 5.0 * rank
    ms = bench.max_over_ranks(mine, world)
    q.put((rank, ms, bench.whole_job_ms_per_step(ms, world)))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, v in got:
        assert ms == 15.0
        assert v == 7.5


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_ms_per_step(3.25, 1) == 3.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_step_sample", lambda *a, **k: called.append(1) or (1.0, "x"))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    assert buf.getvalue() == "" and not called


def test_reference_arm_line_on_rank_zero(monkeypatch):
    import argparse
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "oracle_step_sample", lambda *a, **k: (1234.5, "stub sample"))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(steps=2, warmup=1))
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["value"] == 1234.5
    assert line["unit"] == bench.UNIT and line["higher_is_better"] is False
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["unit"] == bench.UNIT and line["cpu_baseline"]["cores"] == bench.ORACLE_THREADS
    assert "extrapolated" in line["cpu_baseline"]


def test_oracle_step_sample_runs_on_a_small_mesh():
    import bench
    from synthetic import small_cantilever

    v, note = bench.oracle_step_sample(small_cantilever(8, 4, 4), budget_s=0.2)
    assert v is None and "no stored iteration count" in note
