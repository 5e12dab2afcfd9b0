"""The multi-process path of bench.py (one process per GPU, independent
replicas) on CPU with the gloo backend, world size 2: the job time is the
slowest rank's, the job value counts every rank's replica, replicas draw
different seeds, and the reference arm runs on rank 0 alone."""
import io
import os
import sys
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.rank_info()
        ms = 2.0 + 3.0 * rank  # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, w, "cpu")
        out[rank] = (w, r, loc, job_ms, bench.job_value(1000, 3, w, job_ms), bench.replica_seeds(r))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_value_and_seeds():
    world, port = 2, 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (w, r, loc, job_ms, value, seeds) in res.items():
        assert (w, r, loc) == (2, rank, rank)
        assert job_ms == 5.0  # the slowest rank sets the job's time
        assert value == pytest.approx(1000 * 3 * 2 / 5e-3)  # both replicas counted
    assert res[0][5] != res[1][5]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(None)  # returns before touching its arguments
    assert buf.getvalue() == ""
