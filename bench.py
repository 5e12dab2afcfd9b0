"""Throughput benchmark: DOF-updates per second per SSP-RK stage, mixed /
learned variants vs plain FP32 at fixed L1 error.

Headline workload (the largest configuration, one GPU): 256^3 cells, degree
k=3 (20 modes x 4 fields = 1,342,177,280 DOF), SSP-RK3, isothermal cs=1, CFL
0.3, vNR artificial viscosity (alpha=2, beta=0.2), Rusanov faces, OU driving
at Mach 3 (|k| in [1,3], zeta=0.5, seed 0) switched off after one eddy time
T = L/(2 cs M).  The timed state is synthetic developed turbulence: a Gaussian
random velocity field with E(k) ~ k^-2 at rms Mach 3 (seed 105, exact Legendre
coefficients, built on the GPU), rho = 1, relaxed by the method itself (plain
FP32, driven) so that shocks and density contrasts form, then taken as the
state at t = T: the timed steps are the undriven decay.

One step = the whole hot path: CFL dt, and per stage the RHS with viscous
pressure, Riemann fluxes and the stage combine with positivity, and the
velocity projection for the next stage.  L2 is flushed (a 256 MB write)
before every timed step, outside the timed interval (the state, 5.4 GB, is
larger than L2 as well).

Variants: plain FP32, split-BF16 x3 tensor-core products ("x3": tcgen05
kernels), and the learned viscosity sensor (learned-f32, learned-x3; network
trained here, untimed, on plain-sensor pairs of separate driven runs at Mach 3
and Mach 10, seeds 2 and 3, never the evaluation seeds).

Fixed L1 (density, eq. l1_norm):
  precision variants (x3): against an FP64 run of the same mesh from the same
  state with the same dt sequence (recorded by the FP64 run and replayed), as
  is plain FP32;
  learned variants: on the learned-sensor configuration (128^3, k=3, Mach-6
  driven state, seed 104), against the plain scheme on the 2N^3 mesh from the
  exactly prolonged state (2n steps at dt/2), restricted back by L2
  projection; plain FP32 at N against the same reference.
A variant counts when its L1 is within 1.1x of plain FP32's; `value` is the
fastest counting variant.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a 16^3 sub-box at the same degree and scheme).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage, mixed/learned vs plain FP32 at fixed L1 error"
UNIT = "DOF-updates/s"


def workload(args):
    T = 1.0 / (2.0 * args.mach)
    return {"workload": "decaying isothermal turbulence after Mach-%g OU driving switched off at T, %d^3 cells, "
                        "DG k=%d (P%d), SSP-RK3" % (args.mach, args.N, args.k, args.k),
            "N": args.N, "k": args.k, "dof": 4 * ((args.k + 1) * (args.k + 2) * (args.k + 3) // 6) * args.N ** 3,
            "rk_stages": 3, "mach": args.mach, "cs": 1.0, "cfl": 0.3, "av": "vNR alpha=2 beta=0.2",
            "riemann": {"rusanov": "Rusanov", "hll": "HLL", "hllc": "HLLC"}[args.riemann],
            "forcing": "OU |k|<=3 zeta=0.5 seed 0, off after T=%.4f" % T, "diffusion": args.diffusion,
            "state": "synthetic k^-2 velocity (seed 105) relaxed %d driven FP32 steps, taken as the state at t=T"
                     % args.relax,
            "l2": "flushed (256 MB write) before every timed step; state larger than L2",
            "learned_gate": "learned variants: nu/(cs h/p) < %g -> nu = 0 (tiles of 16 such cells skip div v)"
                            % args.nu_gate}


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


# committed ncu summaries of the stage kernels, per variant: (file, kernel sources)
PROFILE = {"x3": ("k5_stage_x3_64c_k3.md", ("dg_tc5_kernels.cuh", "dg_tc5.cuh", "dg_tc5.cu", "dg_common.cuh")),
           "f32": ("k_tile_f32_stage_64c_k3.md", ("dg_tile.cuh", "dg_mma.cuh", "dg_common.cuh",
                                                   "dg_launch_impl.cuh"))}


def profiled_traffic(variant, N):
    """DRAM bytes per stage from the committed ncu summary of the variant's stage
    kernels (captured at 64^3, scaled by the cells), or None when there is none
    or the kernel sources changed since the capture (their SHA-1 is recorded
    next to the figure)."""
    import hashlib
    import re
    key = variant.split("-")[-1]
    if key not in PROFILE:
        return None
    name, srcs = PROFILE[key]
    f = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(f):
        return None
    txt = open(f).read()
    m_t = re.search(r"traffic_per_stage_bytes:\s*(\d+)", txt)
    m_h = re.search(r"kernel_sources_sha1:\s*([0-9a-f]{40})", txt)
    if not (m_t and m_h):
        return None
    h = hashlib.sha1()
    for name in srcs:
        with open(os.path.join(ROOT, "paper_2401_06841_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != m_h.group(1):
        return None
    return int(m_t.group(1)) * (N / 64) ** 3


def adiabatic_arm(args, dev, seed, flush, world, near_isothermal=False):
    """The five-variable adiabatic system (Sec. 2.1) on the same mesh and
    degree, FP32, steps timed like the main variants (L2 flushed before each,
    CUDA events on the solver's stream).  Default: decaying turbulence at rms
    Mach 0.5, gamma 1.4.  near_isothermal: the paper's way of running driven
    turbulence (Sec. 4.2) -- gamma 1.0001, OU driving at Mach 3, the uniform
    temperature restored after every step, the injected and dissipated
    energies reported.  Algorithmic bytes per DOF and stage: u^(s), u^n (2/3
    on average over the SSP-RK3 stages) and u^(s+1), one word each (+ a_h,
    3/5 word, when driven)."""
    import torch
    from paper_2401_06841_gb300 import AdiabaticSolver
    from paper_2401_06841_gb300 import inputs as I
    N, k, S = args.adi_N, args.k, 3
    b = (k + 1) * (k + 2) * (k + 3) // 6
    dof = 5 * b * N ** 3
    gamma = 1.0001 if near_isothermal else 1.4
    s = AdiabaticSolver(N, k, gamma=gamma, precision="f32", rk_stages=S, device=dev)
    if near_isothermal:
        # reset mode: states carry the energy offset e - rho cs^2/(gamma - 1), formed here in FP64
        s.set_forcing(mach=args.mach, zeta=0.5, seed=seed, cs_ref=1.0)
        s.set_reset(1.0)
        u0 = I.adiabatic_turbulent_state(N, k, seed=seed + 3, mach=1.0, gamma=gamma)
        u0[:, 4] -= 1.0 / (gamma - 1.0) * u0[:, 0]
        s.set_state(u0)
    else:
        s.set_state(I.adiabatic_turbulent_state(N, k, seed=seed + 2, mach=0.5))

    def flush_l2():
        with torch.cuda.stream(s.stream):
            flush.fill_(1.0)

    for _ in range(args.warmup):
        flush_l2()
        s.step(1)
    # totals and energy budget over the timed steps only (the warm-up steps
    # include the first reset of the synthetic start state)
    t0 = s.totals()
    b0 = s.energy_budget()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush_l2()
        starts[i].record(s.stream)
        s.step(1)
        ends[i].record(s.stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(e) for a, e in zip(starts, ends)) / args.steps, world, dev)
    t1 = s.totals()
    b1 = s.energy_budget()
    budget = (b1[0] - b0[0], b1[1] - b0[1])
    s.close()
    hbm, _, src = peaks()
    bytes_stage = dof * 4 * (1 + 2.0 / 3.0 + 1 + (0.6 if near_isothermal else 0.0))
    achieved = bytes_stage / (ms / S * 1e-3) / 1e9
    if near_isothermal:
        wl = ("driven near-isothermal turbulence, %d^3 cells, DG k=%d, SSP-RK3, gamma 1.0001 with the "
              "uniform-temperature reset, OU Mach %g (five variables)" % (N, k, args.mach))
    else:
        wl = "decaying turbulence, %d^3 cells, DG k=%d, SSP-RK3, rms Mach 0.5, gamma 1.4 (five variables)" % (N, k)
    out = {"workload": wl,
            "value": job_value(dof, S, world, ms), "unit": UNIT, "ms_per_step": ms, "dtype": "f32", "dof": dof,
            "launches_per_step": S + 1 + (1 if near_isothermal else 0),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_source": src, "bytes_per_stage": bytes_stage,
                         "timed": "whole stages (projection + stage kernel)"},
            "relative_drift": {"mass": (t1["mass"] - t0["mass"]) / t0["mass"],
                               "energy": (t1["energy"] - t0["energy"]) / t0["energy"]},
            "p_min": t1["p_min"], "rho_min": t1["rho_min"]}
    if near_isothermal:
        out["energy_budget_timed_steps"] = {"injected": budget[0], "dissipated": budget[1],
                                            "kinetic_change": t1["ekin"] - t0["ekin"]}
    return out


def cpu_model():
    """The host CPU's model name (lscpu), or the platform's processor string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_arm(args, steps, warmup, threads=0):
    """FP64 CPU oracle on a bounded sample: a 16^3 box at the workload's degree,
    the undriven decay of a synthetic turbulent state (as the timed GPU steps),
    on `threads` host threads (0: all cores; OpenMP over cells, the interface
    loop in parity colours)."""
    from oracle import oracle as O
    from paper_2401_06841_gb300 import inputs as I
    used = O.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    n = args.sample_N
    cfg = O.make_cfg(n, args.k, rk_stages=3, riemann=args.riemann, eps_diff=args.diffusion)
    u = I.turbulent_state(n, args.k, seed=102, mach=args.mach)
    t = 0.0
    for _ in range(warmup):
        rc, t, _, _ = O.run(cfg, u, 1, t=t)
    t0 = time.perf_counter()
    for _ in range(steps):
        rc, t, _, _ = O.run(cfg, u, 1, t=t)
        assert rc == 0
    wall = time.perf_counter() - t0
    dofs = 4 * O.nmodes(args.k) * n ** 3
    value = dofs * 3 * steps / wall
    return value, wall, {"kind": "oracle", "cores": used, "cpu": cpu_model(), "nproc": os.cpu_count(),
                         "sample": "%d^3 cells at k=%d, SSP-RK3, undriven decay, %d steps (FP64 C, %d thread%s)"
                                   % (n, args.k, steps, used, "" if used == 1 else "s")}


def adiabatic_oracle_arm(args, near_isothermal, steps=2):
    """The adiabatic oracle on a bounded sample: 16^3 cells at the workload's
    degree, the same kind of state (and driving with the reset), FP64 C."""
    from oracle import oracle as O
    from paper_2401_06841_gb300 import inputs as I
    n = args.sample_N
    cfg = O.make_cfg(n, args.k, rk_stages=3)
    if near_isothermal:
        g, cs = 1.0001, 1.0
        u = I.adiabatic_turbulent_state(n, args.k, seed=103, mach=1.0, gamma=g)
        fo = O.Forcing(mach=args.mach, zeta=0.5, seed=0, cs=cs)
    else:
        g, cs, fo = 1.4, 0.0, None
        u = I.adiabatic_turbulent_state(n, args.k, seed=102, mach=0.5)
    t0 = time.perf_counter()
    rc, _, _, _, _ = O.adi_run_driven(cfg, g, cs, u, steps, forcing=fo)
    wall = time.perf_counter() - t0
    assert rc == 0
    dofs = 5 * O.nmodes(args.k) * n ** 3
    return {"kind": "oracle", "cores": 1, "unit": UNIT, "value": dofs * 3 * steps / wall,
            "sample": "%d^3 cells at k=%d, SSP-RK3, %d steps of the same workload (single-threaded FP64 C)"
                      % (n, args.k, steps)}


# ---- one process per GPU (torchrun): independent replicas, no data-path collective ----
def rank_info():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms, world, device):
    """The slowest rank's time per step (the job's time): all-reduce MAX."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(dof, stages, world, ms):
    """Whole-job DOF-updates/s per stage: every rank advances its own replica
    of dof unknowns by `stages` stages per step in ms milliseconds."""
    return dof * stages * world / (ms * 1e-3)


def replica_seeds(rank):
    """(initial-state seed, forcing seed) of a rank's replica."""
    return 102 + rank, rank


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


def train_sensor(args, dev):
    """The learned sensor's network, trained (untimed) on plain-sensor pairs of
    separate driven runs: Mach 3 (seed 2) and Mach 10 (seed 3) at k=3, snapshots
    every 10 steps, AV-active and inactive cells balanced 1:1."""
    import torch
    from paper_2401_06841_gb300 import Solver
    from paper_2401_06841_gb300 import inputs as I
    N, k = args.train_N, args.k
    b = (k + 1) * (k + 2) * (k + 3) // 6
    trainer = Solver(N, k, precision="f32", av="learned", device=dev, riemann=args.riemann)
    trainer.set_av_weights(I.mlp_init(2 * b, seed=1))
    xs, ys = [], []
    for mach, seed in ((3.0, 2), (10.0, 3)):
        run = Solver(N, k, precision="f32", rk_stages=3, device=dev, riemann=args.riemann)
        run.set_state(I.turbulent_state_device(N, k, seed=seed, mach=mach, device=dev))
        run.set_forcing(mach=mach, zeta=0.5, seed=seed)
        for i in range(30):
            _, dtl = run.step(1)
            if i % 10 == 9:
                trainer.set_state(run.get_state())
                x, y = trainer.generate_pairs(dtl)
                xs.append(x)
                ys.append(y)
        run.close()
    X, Y = torch.cat(xs), torch.cat(ys)
    g = torch.Generator(device=X.device).manual_seed(0)
    floor = float(Y.min())
    act = torch.nonzero(Y > floor + 1e-3).flatten()
    ina = torch.nonzero(Y <= floor + 1e-3).flatten()
    ina = ina[torch.randperm(len(ina), device=X.device, generator=g)[: max(len(act), 1)]]
    sel = torch.cat([act, ina])
    sel = sel[torch.randperm(len(sel), device=X.device, generator=g)]
    t0 = time.perf_counter()
    loss = trainer.mlp_train(X[sel], Y[sel], epochs=args.train_epochs, batch=4096, lr=2e-3)
    info = {"pairs": int(len(sel)), "active": int(len(act)), "epochs": args.train_epochs, "batch": 4096,
            "final_loss": loss, "seconds": time.perf_counter() - t0,
            "runs": "k=%d %d^3 driven Mach 3 (seed 2) and Mach 10 (seed 3), snapshots every 10 steps" % (k, N)}
    w = trainer.get_av_weights()
    trainer.close()
    return w, info


def make_solver(v, N, k, args, dev, weights):
    from paper_2401_06841_gb300 import Solver
    prec = v.split("-")[-1]
    learned = v.startswith("learned")
    s = Solver(N, k, precision=prec, rk_stages=3, av="learned" if learned else "vnr", device=dev,
               riemann=args.riemann, diffusion=args.diffusion, fused_infer="-fused-" in v,
               x3_backend=args.x3_backend, nu_gate=args.nu_gate if learned else 0.0)
    if v.startswith("learned"):
        s.set_av_weights(weights)
    return s


def time_variant(v, S0, meta0, args, dev, weights, flush, world):
    import torch
    N, k = args.N, args.k
    b = (k + 1) * (k + 2) * (k + 3) // 6
    dof = 4 * b * N ** 3
    s = make_solver(v, N, k, args, dev, weights)
    s.set_forcing(mach=args.mach, zeta=0.5, seed=0, t_off=1.0 / (2.0 * args.mach))
    s.set_state(S0)
    s.set_meta(meta0)
    stream = s.stream

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    for _ in range(args.warmup):
        flush_l2()
        s.step(1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    s.profile(True)
    for i in range(args.steps):
        flush_l2()
        starts[i].record(stream)
        s.step(1)
        ends[i].record(stream)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    per_step = sorted(a.elapsed_time(e) for a, e in zip(starts, ends))
    ms = max_over_ranks(sum(per_step) / args.steps, world, dev)
    n_st = max(prof["n_rhs"], 1)
    stage_ms = (prof["ms_rhs"] + prof["ms_project"]) / n_st
    out = {"value": job_value(dof, 3, world, ms), "ms_per_step": ms, "step_ms_best": per_step[0],
           "step_ms_median": per_step[len(per_step) // 2], "stage_ms": stage_ms,
           "rhs_kernels_ms": prof["ms_rhs"] / n_st, "projection_ms": prof["ms_project"] / n_st,
           "other_ms_per_step": (prof["ms_other"] + prof["ms_force"]) / args.steps,
           "launches": int(prof["launches"]), "launches_per_step": prof["launches"] / args.steps,
           "gated_tile_frac": prof["tiles_gated"] / max(prof["tiles_volume"], 1)}
    return s, out


def precision_gate(variants, S0, meta0, args, dev):
    """L1 density error of the precision variants and of plain FP32 against an FP64
    run of the same mesh from the same state, the FP64 run's dt sequence replayed."""
    from paper_2401_06841_gb300 import Solver
    N, k = args.N, args.k
    T = 1.0 / (2.0 * args.mach)
    ref = Solver(N, k, precision="f64", rk_stages=3, device=dev, riemann=args.riemann, diffusion=args.diffusion)
    ref.set_forcing(mach=args.mach, zeta=0.5, seed=0, t_off=T)
    ref.set_state(S0.double())
    ref.set_meta(meta0)
    dts = []
    t0 = time.perf_counter()
    for _ in range(args.l1_steps):
        _, d = ref.step(1)
        dts.append(d)
    ref_s = time.perf_counter() - t0
    R = ref.get_state()
    out = {}
    for v in ["f32"] + [v for v in variants if not v.startswith("learned") and v != "f32"]:
        s = make_solver(v, N, k, args, dev, None)
        s.set_forcing(mach=args.mach, zeta=0.5, seed=0, t_off=T)
        s.set_state(S0)
        s.set_meta(meta0)
        for d in dts:
            s.step(1, fixed_dt=d)
        out[v] = ref.l1_density(s.get_state().double(), R)
        s.close()
    ref.close()
    return out, {"reference": "FP64 GPU run, same mesh and state, dt sequence replayed", "steps": args.l1_steps,
                 "dt": dts, "reference_seconds": ref_s}


def learned_gate(variants, args, dev, weights):
    """The learned-sensor configuration (N_l^3, k=3, Mach-6 OU-driven turbulence,
    seed 104): plain and learned variants stepped from the same driven state with
    the driving continued (same OU state) and the same dt, each timed, and their
    density L1 error against the plain FP32 scheme on the 2N_l^3 mesh from the
    exactly prolonged state (driven likewise)."""
    import torch
    from paper_2401_06841_gb300 import Solver
    from paper_2401_06841_gb300 import inputs as I
    from paper_2401_06841_gb300 import transfer as Tr
    N, k = args.l_N, args.k
    b = (k + 1) * (k + 2) * (k + 3) // 6
    n = args.l1_steps_learned
    base = Solver(N, k, precision="f32", rk_stages=3, device=dev, riemann=args.riemann)
    base.set_state(I.turbulent_state_device(N, k, seed=104, mach=6.0, device=dev))
    base.set_forcing(mach=6.0, zeta=0.5, seed=4)
    base.step(args.l_relax)
    S4 = base.get_state().clone()
    meta4 = base.get_meta()
    diag = {k_: v for k_, v in base.diagnostics().items() if k_ in ("mach", "rho_min", "rho_max", "av_frac")}
    dt = 0.8 * 0.3 * (1.0 / N) / ((k + 1) * base.diagnostics()["max_speed"])
    base.close()
    fine = Solver(2 * N, k, precision="f32", rk_stages=3, device=dev, riemann=args.riemann)
    fine.set_forcing(mach=6.0, zeta=0.5, seed=4)
    fine.set_state(Tr.prolong(S4, N, k))
    fine.set_meta(meta4)
    fine.step(2 * n, fixed_dt=dt / 2)
    ref = Tr.restrict(fine.get_state(), N, k).contiguous()
    fine.close()
    out, timing = {}, {}
    names = ["f32"] + (["x3"] if any(v.endswith("x3") for v in variants) else []) + \
        [v for v in variants if v.startswith("learned")]
    for v in names:
        s = make_solver(v, N, k, args, dev, weights)
        s.set_forcing(mach=6.0, zeta=0.5, seed=4)
        s.set_state(S4)
        s.set_meta(meta4)
        s.step(1, fixed_dt=dt)  # warm-up (and the first learned coefficient)
        s.set_state(S4)
        s.set_meta(meta4)
        torch.cuda.synchronize()
        s.profile(True)
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(s.stream)
        s.step(n, fixed_dt=dt)
        b_ev.record(s.stream)
        torch.cuda.synchronize()
        prof = s.profile_read()
        ms = a_ev.elapsed_time(b_ev) / n
        out[v] = s.l1_density(s.get_state(), ref)
        timing[v] = {"value": 3 * 4 * b * N ** 3 / (3 * ms * 1e-3), "ms_per_step": ms,
                     "gated_tile_frac": prof["tiles_gated"] / max(prof["tiles_volume"], 1), "l1_rho": out[v]}
        s.close()
    return out, {"reference": "plain FP32 on the 2N^3 mesh from the prolonged state (2n steps at dt/2), "
                              "restricted by L2 projection; every run driven on (the relaxation's OU state)",
                 "mesh": N, "steps": n, "dt": dt, "diag_start": diag,
                 "state": "synthetic k^-2 velocity, Mach 6 (seed 104), %d driven steps" % args.l_relax,
                 "timing": timing, "unit": UNIT}


def config3_arm(args, dev):
    """The strong-shock configuration: 128^3 cells (--c3-N), k=2, SSP-RK3, FP32,
    plain sensor and projection, driven towards Mach 10 by solenoidal OU forcing
    (seed 1) from rho = 1, v = 0; training pairs generated from the state every
    50 steps.  Timed: c3-steps steps (L2 not flushed: the run as a run) with the
    pair generations they contain."""
    import torch
    from paper_2401_06841_gb300 import Solver
    N, k = args.c3_N, 2
    b = (k + 1) * (k + 2) * (k + 3) // 6
    s = Solver(N, k, precision="f32", rk_stages=3, av="vnr", device=dev, riemann=args.riemann)
    pairs = Solver(N, k, precision="f32", av="learned", device=dev, riemann=args.riemann)
    u0 = torch.zeros(N ** 3, 4, b, dtype=torch.float32, device=dev)
    u0[:, 0, 0] = 1.0
    s.set_state(u0)
    s.set_forcing(mach=10.0, zeta=1.0, seed=1)
    s.step(3)
    torch.cuda.synchronize()
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_ev.record(s.stream)
    npairs = 0
    for i in range(args.c3_steps):
        _, dt = s.step(1)
        if (i + 4) % 50 == 0:
            pairs.set_state(s.get_state())
            x, y = pairs.generate_pairs(dt)
            npairs += int(y.numel())
    b_ev.record(s.stream)
    torch.cuda.synchronize()
    ms = a_ev.elapsed_time(b_ev) / args.c3_steps
    d = s.diagnostics()
    s.close()
    pairs.close()
    return {"workload": "driven to Mach 10 (solenoidal OU, seed 1) from rest, %d^3 cells, DG k=2 (P2), SSP-RK3, "
                        "FP32, plain vNR sensor; pairs every 50 steps" % N,
            "value": 3 * 4 * b * N ** 3 / (3 * ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": args.c3_steps, "warmup": 3, "pairs": npairs,
            "state_after": {k_: d[k_] for k_ in ("mach", "rho_min", "rho_max", "av_frac")}}


def driven_start_arm(args, dev):
    """Mach-3 OU driving from rest (rho = 1, v = 0; zeta 0.5, seed 11), --start-N^3
    cells, k=2, SSP-RK3, FP32, in both positivity modes (Sec. 3.1): the rescaling
    of the stage outputs, run until it fails or reaches the end time, and the
    repetition of troubled steps, run to --start-t.  Reports how far each got,
    the repeated attempts (flatten launches) and the state at the end."""
    import math
    import torch
    from paper_2401_06841_gb300 import Solver
    from paper_2401_06841_gb300 import _lib as B
    N, k, t_end = args.start_N, 2, args.start_t
    b = (k + 1) * (k + 2) * (k + 3) // 6
    out = {"workload": "Mach-3 OU driving (zeta 0.5, seed 11) from rho = 1, v = 0, %d^3 cells, DG k=2 (P2), "
                       "SSP-RK3, FP32, to t = %g" % (N, t_end)}
    u0 = torch.zeros(N ** 3, 4, b, dtype=torch.float32, device=dev)
    u0[:, 0, 0] = 1.0
    for pos in ("scale", "repeat"):
        s = Solver(N, k, precision="f32", rk_stages=3, av="vnr", device=dev, positivity=pos)
        s.set_state(u0)
        s.set_forcing(mach=3.0, zeta=0.5, seed=11)
        s.profile(True)
        t, steps, err = 0.0, 0, None
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(s.stream)
        try:
            while t < t_end and steps < 200000:
                t, _ = s.step(10)
                steps += 10
                if pos == "scale" and steps % 100 == 0 and not (s.diagnostics()["max_speed"] < 1e3):
                    err = "wave speed above 1e3 cs"
                    break
        except B.DGError as e:
            err = str(e)
        b_ev.record(s.stream)
        torch.cuda.synchronize()
        ms = a_ev.elapsed_time(b_ev)
        prof = s.profile_read()
        d = s.diagnostics()
        s.close()
        out[pos] = {"t_reached": t, "steps": steps, "failed": err, "wall_s": ms * 1e-3,
                    "flatten_launches": int(prof["n_other"]) if pos == "repeat" else 0,
                    "state_at_end": {k_: (d[k_] if math.isfinite(d[k_]) else None)
                                     for k_ in ("mach", "rho_min", "rho_max", "max_speed")}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--mach", type=float, default=3.0)
    ap.add_argument("--relax", type=int, default=30)
    ap.add_argument("--sample-N", dest="sample_N", type=int, default=16)
    ap.add_argument("--cpu-steps", dest="cpu_steps", type=int, default=4)
    ap.add_argument("--l1-steps", dest="l1_steps", type=int, default=3,
                    help="steps of the FP64 same-mesh reference (precision variants)")
    ap.add_argument("--l-N", dest="l_N", type=int, default=128, help="mesh of the learned-sensor configuration")
    ap.add_argument("--l-relax", dest="l_relax", type=int, default=20)
    ap.add_argument("--l1-steps-learned", dest="l1_steps_learned", type=int, default=10)
    ap.add_argument("--train-N", dest="train_N", type=int, default=64)
    ap.add_argument("--adi-N", dest="adi_N", type=int, default=64)
    ap.add_argument("--variants", default="f32,x3,learned-f32,learned-x3",
                    help="comma list of f32, x3, learned-f32, learned-x3, learned-fused-f32, learned-fused-x3 "
                         "(fused: the sensor network evaluated in the last stage's kernel)")
    ap.add_argument("--no-cpu", dest="no_cpu", action="store_true")
    ap.add_argument("--no-l1", dest="no_l1", action="store_true")
    ap.add_argument("--riemann", default="rusanov", choices=["rusanov", "hll", "hllc"])
    ap.add_argument("--train-epochs", dest="train_epochs", type=int, default=20)
    ap.add_argument("--diffusion", type=float, default=0.0, help="eps of an added div(eps grad u)")
    ap.add_argument("--x3-backend", dest="x3_backend", default="tcgen05", choices=["tcgen05", "mma"],
                    help="order-3 x3 stage: the tcgen05 kernels or the fused mma.sync kernel")
    ap.add_argument("--c3-N", dest="c3_N", type=int, default=128, help="mesh of the strong-shock configuration")
    ap.add_argument("--c3-steps", dest="c3_steps", type=int, default=100)
    ap.add_argument("--no-c3", dest="no_c3", action="store_true")
    ap.add_argument("--start-N", dest="start_N", type=int, default=64,
                    help="mesh of the driven start from rest in both positivity modes")
    ap.add_argument("--start-t", dest="start_t", type=float, default=0.2)
    ap.add_argument("--no-start", dest="no_start", action="store_true")
    ap.add_argument("--nu-gate", dest="nu_gate", type=float, default=1.0,
                    help="learned variants: cells with nu/(cs h/p) below this get no viscous pressure, and "
                         "tiles of 16 such cells skip div v")
    ap.add_argument("--no-adiabatic", dest="no_adiabatic", action="store_true",
                    help="skip the timing of the five-variable adiabatic system")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world, rank, local = rank_info()
    state_seed, force_seed = replica_seeds(rank)
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    from paper_2401_06841_gb300 import Solver
    from paper_2401_06841_gb300 import inputs as I

    N, k = args.N, args.k
    b = (k + 1) * (k + 2) * (k + 3) // 6
    S = 3
    dof = 4 * b * N ** 3
    T = 1.0 / (2.0 * args.mach)
    variants = [v for v in args.variants.split(",") if v]
    # ---- the learned sensor: trained first, on runs of its own seeds (untimed) ----
    weights, training = (None, None)
    if any(v.startswith("learned") for v in variants):
        weights, training = train_sensor(args, dev)
    # ---- the timing state: synthetic turbulence relaxed by the driven method, then
    # taken as the state at t = T (driving off from the first timed step on) ----
    base = Solver(N, k, precision="f32", rk_stages=S, device=dev, riemann=args.riemann, diffusion=args.diffusion)
    base.set_state(I.turbulent_state_device(N, k, seed=state_seed + 3, mach=args.mach, device=dev))
    base.set_forcing(mach=args.mach, zeta=0.5, seed=force_seed, t_off=T)
    base.step(args.relax)
    S0 = base.get_state().clone()
    meta0 = base.get_meta()
    meta0.t = T * (1.0 + 1e-9)
    diag0 = {k_: v for k_, v in base.diagnostics().items() if k_ in ("mach", "rho_min", "rho_max", "av_frac")}
    base.close()
    del base

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    clocks = Clocks(local)
    res = {}
    clocks.start()
    time.sleep(0.2)
    for v in variants:
        s, res[v] = time_variant(v, S0, meta0, args, dev, weights, flush, world)
        s.close()
    clk = clocks.stop()

    # ---- fixed L1 error ----
    gates = {}
    if not args.no_l1:
        l1p, ginfo = precision_gate(variants, S0, meta0, args, dev)
        gates["precision"] = dict(ginfo, l1=l1p)
        for v, l1 in l1p.items():
            if v in res:
                res[v]["l1_rho"] = l1
                res[v]["at_fixed_l1"] = l1 <= 1.1 * l1p["f32"]
        if any(v.startswith("learned") for v in variants):
            l1l, linfo = learned_gate(variants, args, dev, weights)
            gates["learned"] = dict(linfo, l1=l1l)
            for v in variants:
                if v.startswith("learned"):
                    res[v]["l1_rho"] = l1l[v]
                    res[v]["l1_rho_plain_f32"] = l1l["f32"]
                    res[v]["at_fixed_l1"] = l1l[v] <= 1.1 * l1l["f32"]
    else:
        for v in variants:
            res[v]["l1_rho"] = None
            res[v]["at_fixed_l1"] = v == "f32"

    counting = [v for v in variants if res[v]["at_fixed_l1"]]
    head = max(counting, key=lambda v: res[v]["value"]) if counting else variants[0]
    r = res[head]
    # roofline of the stage (all its launches): algorithmic bytes per DOF and stage
    # (SSP-RK3 average): u^(s) 1 word + u^n 2/3 word + u^(s+1) 1 word (undriven: no a_h)
    bytes_per_stage = dof * 4 * (1 + 2.0 / 3.0 + 1)
    hbm, bf16, src = peaks()
    achieved = bytes_per_stage / (r["stage_ms"] * 1e-3) / 1e9
    tr = profiled_traffic(head, N)
    kern = ("k5_volume + k5_faces + k5_project (tcgen05)" if head.endswith("x3")
            else "k_tile stage (RHS + SSP-RK stage + positivity + next projection)")
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": tr, "kernel": "%s, %s; one launch = one RK stage" % (kern, head), "peak_source": src,
            "stage_ms": r["stage_ms"], "bytes_per_stage": bytes_per_stage}

    # ---- end to end through the C ABI with pinned host buffers: H2D state, one step, D2H state ----
    hs = make_solver(head, N, k, args, dev, weights)
    hs.set_forcing(mach=args.mach, zeta=0.5, seed=0, t_off=T)
    host_in = S0.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_ms = []
    for i in range(max(3, args.steps // 5)):
        hs.set_meta(meta0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs.L.dg_set_state(hs.h, host_in.data_ptr(), 1)
        hs.step(1)
        hs.L.dg_get_state(hs.h, host_out.data_ptr(), 1)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms.sort()
    e2e_v = job_value(dof, S, world, max_over_ranks(e2e_ms[len(e2e_ms) // 2], world, dev))
    nbytes = host_in.numel() * host_in.element_size()
    del host_in, host_out

    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "x3": "bf16x3+f32"}[head.split("-")[-1]], "data": "synthetic",
            "config": dict(workload(args), variant=head), "roofline": roof, "clocks": clk,
            "gpu_launches": int(r["launches"]),
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "variants": {v: {k_: res[v].get(k_) for k_ in ("value", "ms_per_step", "step_ms_best", "step_ms_median",
                                                           "stage_ms", "rhs_kernels_ms", "projection_ms",
                                                           "other_ms_per_step", "launches_per_step", "l1_rho",
                                                           "l1_rho_plain_f32", "at_fixed_l1", "gated_tile_frac")}
                         for v in variants},
            "fixed_l1": gates, "diag_start": diag0}
    if training is not None:
        line["learned_training"] = training
    # turbulence statistics of the headline solver's state after one step:
    # density PDF (200 bins), structure function (100 bins x 1e5 pairs); wall ms per call
    hs.set_state(S0)
    hs.set_meta(meta0)
    hs.step(1)
    ana = {}
    for name, fn in (("density_pdf_ms", lambda: hs.density_pdf(-2.0, 2.0, 200)),
                     ("structure_function_ms", lambda: hs.structure_function(100, 100000, 0))):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        ana[name] = 1e3 * (time.perf_counter() - t0)
    line["analysis"] = ana
    hs.close()
    del hs, S0
    torch.cuda.empty_cache()
    if not args.no_c3:
        line["config3"] = config3_arm(args, dev)
    if not args.no_start:
        line["driven_start"] = driven_start_arm(args, dev)
    if not args.no_adiabatic:
        line["adiabatic"] = adiabatic_arm(args, dev, state_seed, flush, world)
        line["adiabatic_near_isothermal"] = adiabatic_arm(args, dev, state_seed, flush, world, near_isothermal=True)
        if rank == 0 and not args.no_cpu:
            line["adiabatic"]["cpu_baseline"] = adiabatic_oracle_arm(args, False)
            line["adiabatic_near_isothermal"]["cpu_baseline"] = adiabatic_oracle_arm(args, True)
    if rank == 0 and not args.no_cpu:
        v, wall, cb = oracle_arm(args, args.cpu_steps, 1)
        cb["value"] = v
        cb["unit"] = UNIT
        v1, _, cb1 = oracle_arm(args, max(1, args.cpu_steps // 2), 1, threads=1)
        cb["single_thread"] = dict(cb1, value=v1, unit=UNIT)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
