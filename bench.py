"""Throughput benchmark: DOF-updates per second per SSP-RK stage.

Workload (default): 64^3 cells, degree k=3 (20 modes x 4 fields), SSP-RK3,
isothermal cs=1, vNR artificial viscosity (alpha=2, beta=0.2), OU driving at
Mach 3 (zeta=0.5, seed 0).  The timed state is synthetic driven turbulence:
a Gaussian random velocity field with E(k) ~ k^-2 at Mach 3 (seed 102, exact
Legendre coefficients), rho = 1, relaxed by the method itself for a few
untimed steps so that shocks and density contrasts form.

One step = the whole hot path: driving update when due, CFL dt, and per
stage the velocity projection, the RHS with AV, Riemann fluxes, forcing, the
stage combine and the positivity rescaling.  L2 is flushed (a 256 MB write)
before every timed step, outside the timed interval.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a 16^3 sub-box at the same degree and scheme).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage, mixed/learned vs plain FP32 at fixed L1 error"
UNIT = "DOF-updates/s"


def workload(args):
    return {"workload": "driven isothermal turbulence, 64^3 cells, DG k=3 (P3), SSP-RK3, Mach 3",
            "N": args.N, "k": args.k, "rk_stages": 3, "mach": args.mach, "cs": 1.0, "cfl": 0.3,
            "av": "vNR alpha=2 beta=0.2", "riemann": "Rusanov", "forcing": "OU |k|<=3 zeta=0.5 seed 0",
            "state": "synthetic k^-2 velocity (seed 102) relaxed %d steps" % args.relax,
            "l2": "flushed (256 MB write) before every timed step"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def oracle_arm(args, steps, warmup):
    """FP64 CPU oracle on a bounded sample: a 16^3 box at the workload's degree."""
    import numpy as np
    from oracle import oracle as O
    from paper_2401_06841_gb300 import inputs as I
    n = args.sample_N
    cfg = O.make_cfg(n, args.k, rk_stages=3)
    u = I.turbulent_state(n, args.k, seed=102, mach=args.mach)
    fo = O.Forcing(mach=args.mach, zeta=0.5, seed=0)
    t, ahat = 0.0, None
    for _ in range(warmup):
        rc, t, _, ahat = O.run(cfg, u, 1, forcing=fo, t=t, ahat=ahat)
    t0 = time.perf_counter()
    for _ in range(steps):
        rc, t, _, ahat = O.run(cfg, u, 1, forcing=fo, t=t, ahat=ahat)
        assert rc == 0
    wall = time.perf_counter() - t0
    dofs = 4 * O.nmodes(args.k) * n ** 3
    value = dofs * 3 * steps / wall
    return value, wall, {"kind": "oracle", "cores": 1,
                         "sample": "%d^3 cells at k=%d, SSP-RK3, driven, %d steps (single-threaded FP64 C)"
                                   % (n, args.k, steps)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    value, wall, cb = oracle_arm(args, args.steps, args.warmup)
    cb["value"] = value
    cb["unit"] = UNIT
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload(args), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "x3", "f64"])
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--mach", type=float, default=3.0)
    ap.add_argument("--relax", type=int, default=30)
    ap.add_argument("--sample-N", dest="sample_N", type=int, default=16)
    ap.add_argument("--cpu-steps", dest="cpu_steps", type=int, default=4)
    ap.add_argument("--no-cpu", dest="no_cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2401_06841_gb300 import Solver
    from paper_2401_06841_gb300 import inputs as I

    N, k = args.N, args.k
    b = (k + 1) * (k + 2) * (k + 3) // 6
    S = 3
    # independent replica per rank (the path shards into independent problems)
    u0 = I.turbulent_state(N, k, seed=102 + rank, mach=args.mach)
    s = Solver(N, k, precision=args.precision, rk_stages=S, cfl=0.3, device="cuda:%d" % local)
    s.set_state(u0)
    s.set_forcing(mach=args.mach, zeta=0.5, seed=rank)
    s.step(args.relax)
    stream = s.stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=s.device)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    for _ in range(args.warmup):
        flush_l2()
        s.step(1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    s.profile(True)
    for i in range(args.steps):
        flush_l2()
        starts[i].record(stream)
        s.step(1)
        ends[i].record(stream)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(e) for a, e in zip(starts, ends)) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=s.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    dof = 4 * b * N ** 3
    value = dof * S * world / (ms * 1e-3)

    # dominant kernel: RHS + stage update (K_B); algorithmic bytes per DOF per
    # stage averaged over SSP-RK3: u^(s) 1 word + u^n 2/3 word + out 1 word + a_h 3/4 word
    esz = 8 if args.precision == "f64" else 4
    rhs_ms = prof["ms_rhs"] / max(prof["n_rhs"], 1)
    bytes_per_launch = dof * esz * (1 + 2.0 / 3.0 + 1 + 0.75)
    hbm, bf16, src = peaks()
    achieved = bytes_per_launch / (rhs_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": "k_rhs (RHS + SSP-RK stage + positivity)", "peak_source": src,
            "kernel_ms": rhs_ms, "project_ms": prof["ms_project"] / max(prof["n_project"], 1)}

    # end to end through the public API with host buffers: H2D state, one step, D2H state
    host_in = torch.from_numpy(s.get_state().cpu().numpy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_ms = []
    for i in range(max(3, args.steps // 4)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.L.dg_set_state(s.h, host_in.data_ptr(), 1)
        s.step(1)
        s.L.dg_get_state(s.h, host_out.data_ptr(), 1)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms.sort()
    e2e_v = dof * S * world / (e2e_ms[len(e2e_ms) // 2] * 1e-3)
    nbytes = host_in.numel() * host_in.element_size()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"f32": "f32", "x3": "bf16x3+f32", "f64": "f64"}[args.precision],
            "data": "synthetic", "config": workload(args), "roofline": roof, "clocks": clk,
            "gpu_launches": int(prof["launches"]),
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "diag": {k_: v for k_, v in s.diagnostics().items() if k_ in ("mach", "rho_min", "rho_max", "av_frac")}}
    if rank == 0 and not args.no_cpu:
        v, wall, cb = oracle_arm(args, args.cpu_steps, 1)
        cb["value"] = v
        cb["unit"] = UNIT
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
