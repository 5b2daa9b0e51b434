"""The multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1), the job's step time is
the maximum over ranks and the whole-job value counts every rank's replica; the reference arm
runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_info() == (ws, rank, rank)
    ms = bench.job_step_ms(1.0 + 0.5 * rank, dist, "cpu")
    out[rank] = (ms, bench.job_value(ws, 2048 * 2048, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        ms, value = res[rank]
        assert ms == 1.5
        assert value == pytest.approx(2 * 2048 * 2048 / 1.5e-3)


def test_single_process_step_time_is_local():
    import bench

    assert bench.job_step_ms(3.25, None, "cpu") == 3.25
    assert bench.job_value(1, 100, 2.0) == 100 / 2e-3


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(A(), 2, 1) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys, monkeypatch):
    """Rank 0 prints one JSON line with the contract's keys; the all-cores oracle run itself is
    replaced by a stub here (its timing is what the line reports, not what this test checks)."""
    import json

    import bench

    calls = []

    def fake_all(n, steps, modes, budget, procs):
        calls.append((n, steps, procs))
        return 1.0e6, n * n * steps * procs, 0.5

    monkeypatch.setattr(bench, "oracle_all_cores", fake_all)

    class A:
        steps, warmup, gpus = 4, 1, 1

    assert bench.run_reference(A(), 1, 0) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] == 1.0e6 and d["steps"] == 4 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == os.cpu_count() and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]
    # one warm-up call, then the timed call, both on the same sample size and every core
    assert [c[1] for c in calls] == [1, 4] and calls[0][0] == calls[1][0]
    assert all(c[2] == os.cpu_count() for c in calls)


def test_oracle_on_every_core_counts_each_process():
    """The all-cores oracle run: spawned processes each step their own copy of the sample; the
    reported cell-updates are processes x n^2 x steps."""
    import bench

    modes = [(1, 2, 1.0)]
    v, cells, wall = bench.oracle_all_cores(16, 3, modes, None, 2)
    assert cells == 2 * 16 * 16 * 3
    assert v > 0 and wall > 0
