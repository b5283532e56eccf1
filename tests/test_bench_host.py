"""Host logic of bench.py's multi-GPU form (independent replicas, one
process per GPU): the slowest rank sets the time and the whole-job value
counts every replica.  Exercised with world_size-2 gloo process groups on
the CPU; the reference arm runs on rank 0 only."""
import json
import os
import socket
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as td
    td.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    mine = [10.0 + rank, 5.0 * (world - rank), 3.0]
    got = bench.max_over_ranks(td, mine, "cpu")
    td.barrier()
    q.put((rank, got, bench.job_value(world, 64 ** 3, 20, got[0])))
    td.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, val in res:
        assert got == [11.0, 10.0, 3.0]                    # every rank sees the maxima
        assert val == pytest.approx(2 * 64 ** 3 * 20 / 11e-3)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(None, [1.5, 2], "cpu") == [1.5, 2.0]
    assert bench.job_value(1, 512 ** 3, 20, 10.0) == pytest.approx(512 ** 3 * 20 / 0.01)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = SimpleNamespace(steps=1, warmup=3)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


@pytest.mark.slow
def test_reference_arm_line(capsys, monkeypatch):
    calls = []

    def fake_sample(budget_s=12.0, n=96):
        calls.append(n)
        return {"value": 1.0e6, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": "s"}

    monkeypatch.setattr(bench, "cpu_oracle_sample", fake_sample)
    bench.run_reference(SimpleNamespace(steps=2, warmup=3), rank=0, world=2)
    line = json.loads(capsys.readouterr().out)
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] == 1.0e6
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and len(calls) == 5
