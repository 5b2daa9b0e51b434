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
