"""Multi-process replica path of bench.py on the CPU (gloo, world size 2).

The data path has no collective (each rank advances its own instance); the
only exchanges are the barriers around the timed region and the max-over-ranks
of the elapsed time, from which the whole-job rate is formed.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench._dist()
        bench._barrier(got_ws)
        t_ms = 10.0 * (rank + 1)   # rank 1 is the slower one
        t_max = bench._barrier_max(t_ms, got_ws)
        rate = bench._job_rate(5, t_max / 1e3, got_ws)
        out.put((got_rank, got_ws, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_max_and_job_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    for _, _, t_max, rate in res:
        assert t_max == 20.0                      # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 5 / 0.020)   # units of both ranks over that time


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._barrier_max(3.5, 1) == 3.5
    assert bench._job_rate(10, 0.5, 1) == 20.0
