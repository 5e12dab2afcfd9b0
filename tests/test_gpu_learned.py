"""Learned viscosity sensor on the GPU against its FP64 references.

* gradients of the FP32 training kernels vs the hand-written FP64 backprop
  (relative L2 <= 1e-4: FP32 forward/backward with FP64 gradient sums);
* BF16 tensor-core inference vs the FP64 forward (bound derived below);
* features and labels vs the oracle's; the learned-mode RHS vs the oracle's
  RHS with the same per-cell coefficients;
* a GPU training run vs the FP64 optimiser on the same data and order;
* what training gains: held-out sensor error of the trained network against
  the best constant predictor of the same labels.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="no CUDA device")

from oracle import mlp_oracle as M  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2401_06841_gb300 import Solver  # noqa: E402
from paper_2401_06841_gb300 import inputs as I  # noqa: E402


def learned_solver(N, k, prec="f32", seed=5):
    s = Solver(N, k, precision=prec, av="learned")
    th = M.init_params(2 * I.nmodes(k), seed=seed)
    s.set_av_weights(th.astype(np.float32))
    return s, th


@pytest.mark.gpu
@pytest.mark.parametrize("k", [1, 3])
def test_mlp_gradient_matches_fp64_backprop(k):
    D = 2 * I.nmodes(k)
    s, th = learned_solver(4, k)
    th32 = th.astype(np.float32).astype(np.float64)  # the GPU holds the FP32-rounded parameters
    rng = np.random.default_rng(1)
    X = rng.uniform(-1.5, 1.5, size=(1000, D)).astype(np.float32)
    y = rng.normal(-2.0, 1.0, size=1000).astype(np.float32)
    loss, g = s.mlp_grad(X, y)
    lref, gref = M.loss_and_grad(th32, X.astype(np.float64), y.astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(lref, rel=1e-5)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


@pytest.mark.gpu
@pytest.mark.parametrize("k", [2, 3])
def test_bf16_inference_vs_fp64_forward(k):
    D = 2 * I.nmodes(k)
    s, th = learned_solver(4, k, seed=7)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(4096, D)).astype(np.float32)
    y = s.mlp_forward(X).cpu().numpy().astype(np.float64)
    yref = M.forward(th, X.astype(np.float64))
    # inputs, weights and hidden activations are rounded to bf16 (relative
    # error <= 2^-9 each), accumulation is FP32: to first order the output
    # error is below 3 * 2^-9 times the absolute-value network
    # |W3| . |a2| + |W3| . |W2| . |a1| + ... ; evaluate that sum
    W1, b1, W2, b2, W3, b3 = M.unpack(th, D)
    a1 = M.gelu(X @ W1.T + b1)
    a2 = M.gelu(a1 @ W2.T + b2)
    absnet = (np.abs(a2) @ np.abs(W3) + (np.abs(a1) @ np.abs(W2).T) @ np.abs(W3)
              + ((np.abs(X) @ np.abs(W1).T) @ np.abs(W2).T) @ np.abs(W3))
    bound = 3 * 2.0 ** -9 * absnet
    err = np.abs(y - yref)
    print("bf16 inference k=%d max |dy| %.3e, max bound %.3e" % (k, err.max(), bound.max()))
    assert (err <= bound).all()
    # and within 2e-2 in log(nu) for inputs of order one (a 2 % change of nu)
    assert err.max() < 2e-2


@pytest.mark.gpu
@pytest.mark.parametrize("prec,xtol,ytol", [("f64", 1e-6, 1e-5), ("f32", 2e-5, 2e-3)])
def test_features_and_labels_vs_oracle(prec, xtol, ytol):
    N, k = 5, 2
    u = I.random_state(N, k, seed=11, v_rms=1.0)
    s, _ = learned_solver(N, k, prec)
    s.set_state(u)
    dt = 2e-3
    x, y = s.generate_pairs(dt)
    xr, yr = O.av_features(O.make_cfg(N, k), u, dt)
    assert np.abs(x.cpu().numpy() - xr).max() <= xtol * max(1.0, np.abs(xr).max())
    assert np.abs(y.cpu().numpy() - yr).max() <= ytol


@pytest.mark.gpu
@pytest.mark.parametrize("k", [1, 2, 3])
def test_learned_rhs_parity(k):
    N = 5
    u = I.random_state(N, k, seed=60 + k)
    s, _ = learned_solver(N, k, "f64", seed=k)
    s.set_state(u)
    nu = s.av_nu().cpu().numpy().astype(np.float64)
    assert np.isfinite(nu).all() and (nu > 0).all()
    dt = 0.3 * (1 / N) / ((k + 1) * 6.0)
    got = s.rhs(u, None, dt).cpu().numpy()
    ref = O.rhs_nu(O.make_cfg(N, k), u, nu, None, dt)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err


@pytest.mark.gpu
def test_learned_gate_zeroes_the_coefficient_of_quiet_cells():
    # nu_gate: cells whose predicted nu/(cs h/p) falls below the gate get nu = 0
    # (no viscous pressure); the right-hand side equals the oracle's with the
    # gated coefficients
    N, k = 5, 2
    u = I.random_state(N, k, seed=64)
    s0, th = learned_solver(N, k, "f64", seed=2)
    s0.set_state(u)
    nu0 = s0.av_nu().cpu().numpy().astype(np.float64)
    ref_scale = 1.0 * (1.0 / N) / (k + 1)
    gate = float(np.median(nu0 / ref_scale))
    s = Solver(N, k, precision="f64", av="learned", nu_gate=gate)
    s.set_av_weights(th.astype(np.float32))
    s.set_state(u)
    nu = s.av_nu().cpu().numpy().astype(np.float64)
    quiet = nu0 / ref_scale < gate
    assert 0 < quiet.sum() < len(nu)
    assert (nu[quiet] == 0).all() and np.array_equal(nu[~quiet], nu0[~quiet])
    dt = 0.3 * (1 / N) / ((k + 1) * 6.0)
    got = s.rhs(u, None, dt).cpu().numpy()
    ref = O.rhs_nu(O.make_cfg(N, k), u, nu, None, dt)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("prec,backend,tol", [("f64", "tcgen05", 1e-12), ("f32", "tcgen05", 2e-5),
                                              ("x3", "tcgen05", 5e-5), ("x3", "mma", 5e-5)])
def test_gate_skips_the_divergence_of_quiet_tiles(prec, backend, tol, forced):
    # half of the mesh at rest (cells iz < N/2: whole tiles of consecutive cells),
    # the other half random.  The gate sits above the resting cells' coefficient
    # and at the median of the others, so that the resting tiles have no
    # viscous pressure anywhere: the kernels skip their gradient rows and div v.
    # The right-hand side still equals the oracle's with the gated coefficients,
    # and the profile counts the skipped tiles.
    N, k = 8, 3
    u = I.random_state(N, k, seed=71)
    rest = np.arange(N ** 3) // (N * N) < N // 2
    u[rest] = 0.0
    u[rest, 0, 0] = 1.0
    # a random network under which the resting cells' coefficient lies below a
    # quarter of the others (the first such seed)
    ref_scale = (1.0 / N) / (k + 1)
    s0 = Solver(N, k, precision="f64", av="learned")
    s0.set_state(u)
    for seed in range(6, 64):
        th = M.init_params(2 * I.nmodes(k), seed=seed).astype(np.float32)
        s0.set_av_weights(th)
        nu0 = s0.av_nu().cpu().numpy().astype(np.float64) / ref_scale
        v_rest = nu0[rest].max()
        if np.mean(nu0[~rest] > v_rest) > 0.25:
            break
    s0.close()
    assert np.ptp(nu0[rest]) <= 1e-12 * v_rest and np.mean(nu0[~rest] > v_rest) > 0.25
    gate = max(float(v_rest) * (1 + 1e-6), float(np.median(nu0[~rest])))
    s = Solver(N, k, precision=prec, av="learned", nu_gate=gate, x3_backend=backend)
    s.set_av_weights(th)
    s.set_state(u)
    nu = s.av_nu().cpu().numpy().astype(np.float64)
    assert (nu[rest] == 0).all() and (nu[~rest] > 0).any()
    a = None
    if forced:
        fo = O.Forcing(mach=2.0, zeta=0.5, seed=4)
        a = O.forcing_project(O.make_cfg(N, k), fo.kvec(), fo.amplitudes())
    dt = 0.3 * (1 / N) / ((k + 1) * 6.0)
    s.profile(True)
    got = s.rhs(u, a, dt).cpu().numpy()
    p = s.profile_read()
    s.close()
    ref = O.rhs_nu(O.make_cfg(N, k), u, nu, a, dt)
    err = max(np.linalg.norm(got[:, v] - ref[:, v]) / np.linalg.norm(ref[:, v]) for v in range(4))
    assert err < tol, err
    # tiles of 16 consecutive cells: every tile of the resting half is skipped, a tile
    # with a coefficient above zero is not
    assert p["tiles_volume"] >= (N ** 3) // 16
    assert p["tiles_gated"] >= rest.sum() // 16
    assert p["tiles_gated"] < p["tiles_volume"]


@pytest.mark.gpu
def test_gpu_training_follows_fp64_adam():
    k = 2
    D = 2 * I.nmodes(k)
    s, th = learned_solver(4, k, seed=3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(2048, D)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 1.0).astype(np.float32)
    loss_gpu = s.mlp_train(X, y, epochs=3, batch=256, lr=1e-3)
    th_ref = th.astype(np.float32).astype(np.float64)
    hist = M.train(th_ref, X.astype(np.float64), y.astype(np.float64), epochs=3, batch=256, lr=1e-3)
    w = s.get_av_weights().astype(np.float64)
    assert loss_gpu == pytest.approx(hist[-1], rel=2e-3)
    assert np.linalg.norm(w - th_ref) <= 2e-3 * np.linalg.norm(th_ref)
    assert hist[-1] < 0.5 * hist[0]


@pytest.mark.gpu
def test_trained_sensor_beats_constant_predictor_on_held_out_cells():
    # pairs from a driven Mach-3 run with the plain sensor (k=2, 24^3), seeds
    # for training and evaluation kept apart
    N, k = 24, 2
    plain = Solver(N, k, precision="f32", av="vnr")
    learned, th = learned_solver(N, k, "f32", seed=9)
    xs, ys = [], []
    for seed in (2, 3):
        plain.set_state(I.turbulent_state(N, k, seed=seed, mach=3.0))
        plain.set_forcing(mach=3.0, zeta=0.5, seed=seed)
        for _ in range(4):
            _, dt = plain.step(10)
            learned.set_state(plain.get_state())
            x, y = learned.generate_pairs(dt)
            xs.append(x)
            ys.append(y)
    X = torch.cat(xs)
    Y = torch.cat(ys)
    g = torch.Generator(device=X.device).manual_seed(0)
    perm = torch.randperm(len(Y), device=X.device, generator=g)
    X, Y = X[perm], Y[perm]
    untrained = Solver(N, k, precision="f32", av="learned")
    untrained.set_av_weights(th.astype(np.float32))
    loss = learned.mlp_train(X, Y, epochs=25, batch=4096, lr=2e-3)
    # held-out evaluation state: another seed
    plain.set_state(I.turbulent_state(N, k, seed=17, mach=3.0))
    plain.set_forcing(mach=3.0, zeta=0.5, seed=17)
    _, dt = plain.step(30)
    learned.set_state(plain.get_state())
    xe, ye = learned.generate_pairs(dt)
    pred = learned.mlp_forward(xe)
    mae = (pred - ye).abs().mean().item()
    mae_const = (ye - ye.median()).abs().mean().item()
    mae_init = (untrained.mlp_forward(xe) - ye).abs().mean().item()
    print("sensor MAE in log(nu): trained %.3f, best constant %.3f, untrained %.3f, final train loss %.3f"
          % (mae, mae_const, mae_init, loss))
    # the inputs (rho and |v| coefficients) do not carry the sign of div v, so
    # part of the label stays unpredictable; training must still beat the best
    # constant predictor and the untrained network by a quarter
    assert mae < 0.75 * mae_const
    assert mae < 0.75 * mae_init


def _train_k3_sensor(N, dev="cuda"):
    """network trained on plain-sensor pairs of driven k=3 runs at Mach 3 (seed 2)
    and Mach 10 (seed 3), snapshots every 10 steps, active and inactive cells 1:1"""
    k = 3
    trainer, _ = learned_solver(N, k, "f32", seed=1)
    xs, ys = [], []
    for mach, seed in ((3.0, 2), (10.0, 3)):
        run = Solver(N, k, precision="f32", av="vnr")
        run.set_state(I.turbulent_state(N, k, seed=seed, mach=mach))
        run.set_forcing(mach=mach, zeta=0.5, seed=seed)
        for i in range(30):
            _, dt = run.step(1)
            if i % 10 == 9:
                trainer.set_state(run.get_state())
                x, y = trainer.generate_pairs(dt)
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
    trainer.mlp_train(X[sel], Y[sel], epochs=20, batch=2048, lr=2e-3)
    w = trainer.get_av_weights()
    trainer.close()
    return w


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f32", "x3"])
def test_trained_sensor_gains_over_the_plain_sensor(prec):
    # what the network gains over the method without it (Sec. 5 error-cost
    # comparison): on a held-out Mach-6 state (seed 17; training used seeds 2
    # and 3) and against the FP64 plain scheme on the 2N mesh (discretisation
    # error), the gated learned sensor reaches a density L1 no larger than the
    # plain sensor's while a large share of the tiles skips the div v work (half
    # of them on this Mach-6 state at 24^3); same mesh, precision,
    # steps and dt for both
    from paper_2401_06841_gb300 import transfer as Tr
    N, k, n = 24, 3, 10
    w = _train_k3_sensor(N)
    base = Solver(N, k, precision="f32", av="vnr")
    base.set_state(I.turbulent_state(N, k, seed=17, mach=6.0))
    base.set_forcing(mach=6.0, zeta=0.5, seed=17)
    base.step(20)
    S = base.get_state().clone()
    dt = 0.8 * 0.3 * (1.0 / N) / ((k + 1) * base.diagnostics()["max_speed"])
    base.close()
    fine = Solver(2 * N, k, precision="f64", av="vnr")
    fine.set_state(Tr.prolong(S.double(), N, k))
    fine.step(2 * n, fixed_dt=dt / 2)
    ref = Tr.restrict(fine.get_state(), N, k).contiguous()
    fine.close()
    l1, gated = {}, {}
    for v in ("plain", "learned"):
        s = Solver(N, k, precision=prec, av="vnr" if v == "plain" else "learned", nu_gate=1.0 if v == "learned" else 0.0)
        if v == "learned":
            s.set_av_weights(w)
        s.set_state(S)
        s.profile(True)
        s.step(n, fixed_dt=dt)
        p = s.profile_read()
        l1[v] = s.l1_density(s.get_state().double(), ref)
        gated[v] = p["tiles_gated"] / p["tiles_volume"]
        s.close()
    print("density L1 vs FP64 on 2N: plain %.4e, learned %.4e (ratio %.3f); gated tiles %.3f"
          % (l1["plain"], l1["learned"], l1["learned"] / l1["plain"], gated["learned"]))
    assert gated["plain"] == 0.0
    assert gated["learned"] > 0.3
    assert l1["learned"] <= l1["plain"]


@pytest.mark.gpu
@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32", "x3"])
@pytest.mark.parametrize("N,k,gated", [(5, 1, False), (5, 2, True), (5, 3, False), (7, 3, True)])
def test_carried_coefficient_matches_the_inference_kernel(N, k, prec, gated, fused):
    # the coefficient the next learned step uses for the current state: with
    # fused_infer evaluated by the last stage for the state it writes, else by
    # the inference kernel from the |v| projection the last stage carried.
    # Either equals, bit for bit, the inference kernel's on a fresh projection
    # of the same state (same BF16 roundings, products and accumulation
    # orders).  125 and 343 cells leave ragged tiles (16 cells per tile, 32 at
    # k = 1)
    u = I.random_state(N, k, seed=40 + k, v_rms=0.8)
    th = M.init_params(2 * I.nmodes(k), seed=9).astype(np.float32)
    gate = 0.0
    if gated:
        s0 = Solver(N, k, precision=prec, av="learned")
        s0.set_av_weights(th)
        s0.set_state(u)
        s0.step(1)
        nu0 = s0.av_nu().cpu().numpy().astype(np.float64)
        gate = float(np.median(nu0 / ((1.0 / N) / (k + 1))))
    s = Solver(N, k, precision=prec, av="learned", nu_gate=gate, fused_infer=fused)
    s.set_av_weights(th)
    s.set_state(u)
    with pytest.raises(Exception):
        s.av_nu_carried()  # nothing carried before the first step
    s.step(2)
    carried = s.av_nu_carried().cpu().numpy()
    fresh = s.av_nu().cpu().numpy()
    assert np.array_equal(carried, fresh)
    assert (carried > 0).any()
    if gated:
        assert (carried == 0).any()
    with pytest.raises(Exception):
        s.av_nu_carried()  # dg_av_nu recomputed it: the carry is gone


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6), ("x3", 1e-6)])
def test_learned_steps_fused_and_separate_inference(prec, tol):
    # three learned steps in a row with the coefficient evaluated in the last
    # stage (fused_infer) equal, bit for bit, three steps with the separate
    # inference launch on the same stage kernel (in x3 the in-stage evaluation
    # lives in the fused mma.sync kernel); and both stay within rounding of
    # three steps that each start from a freshly set state (projection and
    # inference launched at the start of every step)
    N, k = 6, 3
    u = I.random_state(N, k, seed=77, v_rms=0.8)
    th = M.init_params(2 * I.nmodes(k), seed=11).astype(np.float32)
    runs = []
    for fused in (True, False):
        a = Solver(N, k, precision=prec, av="learned", fused_infer=fused, x3_backend="mma")
        a.set_av_weights(th)
        a.set_state(u)
        a.step(3)
        runs.append(a.get_state().cpu().numpy().astype(np.float64))
    assert np.array_equal(runs[0], runs[1])
    b = Solver(N, k, precision=prec, av="learned", x3_backend="mma")
    b.set_av_weights(th)
    b.set_state(u)
    for _ in range(3):
        b.step(1)
        b.set_state(b.get_state())
    ub = b.get_state().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(runs[0] - ub) <= tol * np.linalg.norm(ub)
