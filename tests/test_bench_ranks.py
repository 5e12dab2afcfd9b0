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
    with mp.get_context("spawn").Manager() as m:
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


def test_reference_arm_prints_the_contract_line():
    # the reference arm (the FP64 oracle on the host cores) at N = 1: one JSON
    # line with the keys the harness reads, its e2e and cpu_baseline mirroring
    # the line's own value
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["workload"]


def test_profiled_traffic_is_dropped_when_the_kernel_changes(tmp_path, monkeypatch):
    # the stage's DRAM bytes come from the ncu summary only while the kernel
    # sources hash to the value recorded beside them; captured at 64^3, scaled by
    # the number of cells
    import hashlib
    import shutil
    name, srcs = bench.PROFILE["x3"]
    csrc = os.path.join("paper_2401_06841_gb300", "csrc")
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / csrc)
    h = hashlib.sha1()
    for src in srcs:
        shutil.copy(os.path.join(ROOT, csrc, src), tmp_path / csrc / src)
        h.update(open(os.path.join(ROOT, csrc, src), "rb").read())
    with open(tmp_path / "profiles" / name, "w") as fh:
        fh.write("traffic_per_stage_bytes: 300000000\nkernel_sources_sha1: %s\n" % h.hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("x3", 64) == 300000000
    assert bench.profiled_traffic("learned-x3", 128) == 8 * 300000000
    assert bench.profiled_traffic("f32", 64) is None  # no summary for that kernel here
    with open(tmp_path / csrc / srcs[0], "a") as fh:
        fh.write("\n")
    assert bench.profiled_traffic("x3", 64) is None
