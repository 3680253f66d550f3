"""Host logic of the multi-GPU benchmark (one independent replica per rank, weak scaling), run as
two gloo ranks on the CPU: max-over-ranks timing, barrier, whole-job aggregation, and the
reference arm printing on rank 0 only."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank  # rank 1 is the slowest replica
        bench.barrier(world)
        worst = bench.max_over_ranks(ms, world)
        out[rank] = (worst, bench.aggregate_mlups(world, 1000, 10, worst))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_and_aggregate():
    port = 29500 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 125.0
    # 2 replicas x 1000 cells x 10 steps in 0.125 s
    assert abs(res[0][1] - 2 * 1000 * 10 / 0.125 / 1e6) < 1e-12


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup = 1, 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    assert buf.getvalue() == ""


def test_reference_arm_line_on_rank_zero(monkeypatch):
    # the oracle timed on a bounded sample: a positive throughput, the keys of the JSON line
    sys.path.insert(0, ROOT)
    import json

    import bench

    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")

    class A:
        steps, warmup = 1, 1

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A())
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0.0
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # one solver built once and warmed up; each timed step advances it by 8 time steps
    assert "one solver" in line["cpu_baseline"]["sample"] and "1 x 8 FP64 steps" in line["cpu_baseline"]["sample"]
    assert abs(line["ms_per_step"] * 1e-3 * line["value"] * 1e6 - 8 * 1024 * 1024) < 1e-6 * 8 * 1024 * 1024
