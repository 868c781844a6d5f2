"""The benchmark's multi-process path on CPU (gloo, two ranks): every rank
gets the slowest rank's time, the job value counts every rank's units over
that time, and the reference arm's non-zero ranks exit without work."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (t, bench.job_value(1000, world, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    times = [0.25, 0.75]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, _free_port(), times, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r][0] == 0.75
        assert res[r][1] == pytest.approx(2 * 1000 / 0.75)


def test_single_rank_is_its_own_time():
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5
    assert bench.job_value(10, 1, 0.5) == 20.0


def test_reference_arm_nonzero_rank_does_no_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference(bench.parse())
    assert buf.getvalue() == ""
