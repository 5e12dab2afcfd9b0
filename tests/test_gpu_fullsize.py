"""Parity at the full mesh sizes of the benchmark configurations.

* 64^3 cells, k = 3 (the benchmarked workload, its launch path: dg_step with
  the fused stage kernels and the carried projection): two driven steps of a
  turbulent state against the whole-mesh oracle.
* 128^3 cells at k = 2 (Mach-10 state and forcing amplitude, vNR sensor) and at k = 3 (learned
  sensor), 256^3 cells at k = 3: the GPU right-hand side against the oracle
  on sampled cells, each computed from its face neighbourhood (the oracle's
  per-cell arithmetic, no whole-mesh pass).  The 256^3 state is a 4 x 4 x 4
  periodic tiling of a 64^3 state built on the device, which adds an exact
  check over every cell: each copy of the tile has the same right-hand side,
  bit for bit (the operator is local; no forcing, dt given).

Tolerances: the right-hand side of a smooth state is a small difference of
large volume and face terms; FP32 shows relative errors of tens of unit
round-offs and the x3 products add their 2^-16 relative error times that
cancellation (the 64^3 right-hand-side test: 3.5e-6 FP32; bounds 1e-5 and
2e-4).  Over two steps the state itself moves by dt L, so its increment is
compared with the same bounds plus the FP32 rounding of the six stored stage
states, 6 * 2^-24 |u| relative to the increment (it dominates for the
density, whose increment is ~1% of rho), and the state with a bound 100x
tighter plus the same storage term.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="no CUDA device")

from oracle import mlp_oracle as M  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2401_06841_gb300 import Solver  # noqa: E402
from paper_2401_06841_gb300 import inputs as I  # noqa: E402

TOL = {"f32": 1e-5, "x3": 2e-4}


def rel_fields(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return np.array([np.linalg.norm(got[:, v] - ref[:, v]) / np.linalg.norm(ref[:, v]) for v in range(ref.shape[1])])


def sample_cells(N, n, seed):
    # random cells plus the corners and edges of the periodic box
    rng = np.random.default_rng(seed)
    c = rng.choice(N ** 3, n, replace=False)
    e = N - 1
    corners = [((z * N) + y) * N + x for x in (0, e) for y in (0, e) for z in (0, e)]
    return np.unique(np.concatenate([c, corners, [N // 2, N * N - 1, N ** 3 // 2]]))


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "x3"])
def test_full_size_driven_steps_64_k3(prec):
    N, k = 64, 3
    # the oracle starts from the FP32 state the GPU holds
    u = I.turbulent_state(N, k, seed=102, mach=3.0).astype(np.float32).astype(np.float64)
    fo = dict(mach=3.0, zeta=0.5, seed=0)
    s = Solver(N, k, precision=prec)
    s.set_state(u)
    s.set_forcing(**fo)
    t_gpu, _ = s.step(2)
    got = s.get_state().cpu().numpy().astype(np.float64)
    ref = u.copy()
    rc, t_ref, _, _ = O.run(O.make_cfg(N, k), ref, 2, forcing=O.Forcing(**fo))
    assert rc == 0
    assert t_gpu == pytest.approx(t_ref, rel=1e-6)  # CFL maximum in FP32
    err_inc = rel_fields(got - u, ref - u)
    err = rel_fields(got, ref)
    store = np.array([6 * 2.0 ** -24 * np.linalg.norm(u[:, v]) / np.linalg.norm(ref[:, v] - u[:, v])
                      for v in range(4)])
    print("64^3 k=3 two driven steps %s: increment %s (storage term %s) state %s" % (prec, err_inc, store, err))
    assert np.all(err_inc < TOL[prec] + store), err_inc
    assert err.max() < TOL[prec] / 100 + 6 * 2.0 ** -24, err


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "x3"])
def test_sampled_rhs_128_k2_mach10_driven(prec):
    N, k = 128, 2
    u = I.turbulent_state(N, k, seed=1, mach=10.0)
    u[:, 0, :] = I.random_state(N, k, seed=5, rho_wiggle=0.3, v_rms=0.0)[:, 0, :]
    cfg = O.make_cfg(N, k)
    # forcing coefficients of driving amplitude (their projection from the OU
    # modes has its own parity test)
    a = 20.0 * I.random_state(N, k, seed=2, v_rms=1.0)[:, 1:, :]
    dt = 0.3 * (1.0 / N) / ((k + 1) * 12.0)
    s = Solver(N, k, precision=prec)
    got = s.rhs(u, a, dt)
    cells = sample_cells(N, 600, seed=3)
    ref = O.rhs_cells(cfg, u, cells, ahat=a, abar=O.forcing_mean(cfg, u, a), dt_pimax=dt)
    err = rel_fields(got[torch.as_tensor(cells, device=got.device)].cpu().numpy(), ref)
    print("128^3 k=2 Mach 10 sampled RHS %s rel-L2 per field %s" % (prec, err))
    assert err.max() < TOL[prec], err


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "x3"])
def test_sampled_rhs_128_k3_learned(prec):
    # learned sensor: the oracle takes the per-cell coefficients the GPU's
    # inference produced for this state
    N, k = 128, 3
    u = I.turbulent_state(N, k, seed=6, mach=6.0)
    u[:, 0, :] = I.random_state(N, k, seed=9, rho_wiggle=0.3, v_rms=0.0)[:, 0, :]
    th = M.init_params(2 * I.nmodes(k), seed=4).astype(np.float32)
    s = Solver(N, k, precision=prec, av="learned")
    s.set_av_weights(th)
    s.set_state(u)
    nu = s.av_nu().cpu().numpy().astype(np.float64)
    assert (nu > 0).all()
    dt = 0.3 * (1.0 / N) / ((k + 1) * 8.0)
    got = s.rhs(u, None, dt)
    cells = sample_cells(N, 600, seed=4)
    ref = O.rhs_cells(O.make_cfg(N, k), u, cells, dt_pimax=dt, nu_cell=nu[cells])
    err = rel_fields(got[torch.as_tensor(cells, device=got.device)].cpu().numpy(), ref)
    print("128^3 k=3 learned sampled RHS %s rel-L2 per field %s" % (prec, err))
    assert err.max() < TOL[prec], err


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "x3"])
def test_sampled_rhs_256_k3_tiled(prec):
    n, T, k = 64, 4, 3
    N = n * T
    base = I.turbulent_state(n, k, seed=12, mach=3.0)
    base[:, 0, :] = I.random_state(n, k, seed=13, rho_wiggle=0.3, v_rms=0.0)[:, 0, :]
    b = base.shape[-1]
    s = Solver(N, k, precision=prec)
    dev = s.device
    ub = torch.as_tensor(base, dtype=s.dtype, device=dev).view(n, n, n, 4, b)
    u = ub.repeat(T, T, T, 1, 1).reshape(N ** 3, 4, b)
    del ub
    dt = 0.3 * (1.0 / N) / ((k + 1) * 6.0)
    got = s.rhs(u, None, dt)
    del u
    # every copy of the tile: the same right-hand side, bit for bit
    g = got.view(T, n, T, n, T, n, 4, b)
    first = g[0, :, 0, :, 0]
    for tz in range(T):
        for ty in range(T):
            for tx in range(T):
                assert torch.equal(g[tz, :, ty, :, tx], first), (tz, ty, tx)
    cells = sample_cells(N, 600, seed=5)
    ref = O.rhs_cells(O.make_cfg(N, k), base, cells, dt_pimax=dt, base_N=n)
    err = rel_fields(got[torch.as_tensor(cells, device=dev)].cpu().numpy(), ref)
    print("256^3 k=3 sampled RHS %s rel-L2 per field %s" % (prec, err))
    assert err.max() < TOL[prec], err
