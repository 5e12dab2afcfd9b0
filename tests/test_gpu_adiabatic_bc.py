"""Boundaries of the adiabatic system on the GPU (outflow, reflective and inflow
faces; the paper's test problems of Sec. 3.1): parity with the oracle on the
same seeded inputs (right-hand side and steps, FP64 to 1e-12, FP32 to 1e-5 /
3e-5), the Shu-Osher problem (a Mach-3 shock into a sinusoidal density field,
inflow and outflow along x) with the shock where the Rankine-Hugoniot speed
puts it, and the Liska-Wendroff implosion (reflective walls in x and y) keeping
its diagonal symmetry, mass and energy."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="no CUDA device")

from oracle import oracle as O  # noqa: E402
from paper_2401_06841_gb300 import AdiabaticSolver  # noqa: E402
from paper_2401_06841_gb300 import inputs as I  # noqa: E402

G = 1.4


def rel_fields(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return np.array([np.linalg.norm(got[:, v] - ref[:, v]) / max(np.linalg.norm(ref[:, v]), 1e-300)
                     for v in range(ref.shape[1])])


def pnorm(m, x):
    c = np.zeros(m + 1)
    c[m] = 1.0
    return math.sqrt(2 * m + 1) * npleg.legval(x, c)


def project_xy(N, k, fn, nq=8):
    """Cell coefficients [N^3][5][b] of conserved fields fn(x, y) -> (rho, m_x,
    m_y, m_z, e) on [0, 1]^2 (uniform in z): Gauss projection per (ix, iy) cell
    with nq points per axis onto the modes of z-degree 0."""
    xg, wg = np.polynomial.legendre.leggauss(nq)
    deg = I.mode_degrees(k)
    b = len(deg)
    out = np.zeros((N ** 3, 5, b))
    X = (np.arange(N)[:, None] + 0.5 * (xg[None, :] + 1.0)) / N          # [cell][point]
    Pm = np.array([pnorm(m, xg) for m in range(k + 1)])                     # [m][point]
    for iy in range(N):
        for ix in range(N):
            xx, yy = np.meshgrid(X[ix], X[iy], indexing="ij")                # [px][py]
            F = np.asarray(fn(xx, yy))                                       # [5][px][py]
            coef = np.zeros((5, b))
            for l, (i, j, m) in enumerate(deg):
                if m:
                    continue
                wgt = np.outer(wg * Pm[i], wg * Pm[j]) / 4.0                 # (1/4) int int over [-1,1]^2
                coef[:, l] = (F * wgt[None]).sum(axis=(1, 2))
            for iz in range(N):
                out[(iz * N + iy) * N + ix] = coef
    return out


def cons(rho, vx, vy, p):
    return np.array([rho, rho * vx, rho * vy, 0.0 * rho, p / (G - 1) + 0.5 * rho * (vx * vx + vy * vy)])


BCS = ("inflow", "reflect", "outflow")
W_IN = (1.2, 0.5, 0.1, -0.2, 1.4)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("k,riemann", [(1, "rusanov"), (2, "hllc"), (3, "rusanov")])
def test_boundary_rhs_parity(prec, k, riemann):
    N = 5
    u = I.random_energy_state(N, k, seed=40 + k, v_rms=0.3, p_mean=5.0, gamma=G)
    cfg = O.make_cfg(N, k, riemann=riemann, bc=BCS, inflow=W_IN)
    ref = O.adi_rhs(cfg, G, u, 1e-3)
    s = AdiabaticSolver(N, k, gamma=G, precision=prec, riemann=riemann, bc=BCS, inflow=W_IN)
    got = s.rhs(u, 1e-3).cpu().numpy()
    s.close()
    err = rel_fields(got, ref)
    assert err.max() < {"f64": 1e-12, "f32": 1e-5}[prec], err


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_boundary_steps_parity(prec):
    N, k = 5, 2
    u = I.random_energy_state(N, k, seed=77, v_rms=0.3, p_mean=5.0, gamma=G)
    cfg = O.make_cfg(N, k, bc=("reflect", "inflow", "outflow"), inflow=W_IN)
    ref = u.copy()
    rc, t_ref, _ = O.adi_run(cfg, G, ref, 3)
    assert rc == 0
    s = AdiabaticSolver(N, k, gamma=G, precision=prec, bc=("reflect", "inflow", "outflow"), inflow=W_IN)
    s.set_state(u)
    t, _ = s.step(3)
    got = s.get_state().cpu().numpy()
    s.close()
    assert t == pytest.approx(t_ref, rel=1e-13 if prec == "f64" else 1e-6)
    err = rel_fields(got, ref)
    assert err.max() < {"f64": 1e-12, "f32": 3e-5}[prec], err


@pytest.mark.gpu
def test_shu_osher_shock_position():
    # Sec. 3.1: x in [-5, 5] scaled to [0, 1] (t scaled alike); the Mach-3 shock
    # starts at x = -4 and runs into rho = 1 + 0.2 sin(5x) at the speed
    # 3 sqrt(1.4) of a Mach-3 shock into rho = 1, p = 1: at t = 1.8 near x = 2.39
    N, k = 60, 2
    rL, vL, pL = 3.857143, 2.629369, 10.33333

    def fn(x, y):
        X = 10.0 * x - 5.0
        left = X < -4.0
        rho = np.where(left, rL, 1.0 + 0.2 * np.sin(5.0 * X))
        v = np.where(left, vL, 0.0)
        p = np.where(left, pL, 1.0)
        return cons(rho, v, 0.0 * v, p)

    u = project_xy(N, k, fn)
    s = AdiabaticSolver(N, k, gamma=G, precision="f32", bc=("inflow", "periodic", "periodic"),
                        inflow=(rL, vL, 0.0, 0.0, pL))
    s.set_state(u)
    t = 0.0
    while t < 0.18:
        t, dt = s.step(1)
    got = s.get_state().cpu().numpy()
    s.close()
    assert np.isfinite(got).all() and t < 0.181
    rho_mean = got[:N, 0, 0]                        # the row (ix, 0, 0)
    behind = np.nonzero(rho_mean > 2.0)[0]
    x_shock = 10.0 * (behind.max() + 1.0) / N - 5.0  # downstream edge of the last compressed cell
    x_rh = -4.0 + 3.0 * math.sqrt(G) * 10.0 * t
    assert abs(x_shock - x_rh) < 0.4, (x_shock, x_rh)
    # post-shock entropy waves: densities up to about 4.7 behind the shock
    assert 3.5 < rho_mean[: behind.max()].max() < 5.2


@pytest.mark.gpu
def test_implosion_keeps_its_symmetry():
    # Sec. 3.1 (Liska-Wendroff): [0, 0.3]^2 scaled to [0, 1]^2, reflective walls,
    # rho = 0.125, p = 0.14 below the diagonal x + y = 0.5, rho = p = 1 above
    N, k = 48, 1

    def fn(x, y):
        low = x + y < 0.5
        rho = np.where(low, 0.125, 1.0)
        p = np.where(low, 0.14, 1.0)
        return cons(rho, 0.0 * x, 0.0 * x, p)

    u = project_xy(N, k, fn)
    s = AdiabaticSolver(N, k, gamma=G, precision="f32", bc=("reflect", "reflect", "periodic"))
    s.set_state(u)
    tot0 = s.totals()
    t = 0.0
    while t < 0.3:
        t, _ = s.step(10)
    tot1 = s.totals()
    got = s.get_state().cpu().numpy()
    s.close()
    assert np.isfinite(got).all()
    assert abs(tot1["mass"] - tot0["mass"]) < 1e-5 * tot0["mass"]
    assert abs(tot1["energy"] - tot0["energy"]) < 1e-5 * tot0["energy"]
    # mirror about the diagonal: cell (ix, iy) <-> (iy, ix), v_x <-> v_y
    r = got[: N * N].reshape(N, N, 5, -1)           # [iy][ix][var][mode], z-layer 0
    rho = r[:, :, 0, 0]
    assert np.abs(rho - rho.T).max() < 1e-4 * rho.max()
    assert np.abs(r[:, :, 1, 0] - r[:, :, 2, 0].T).max() < 1e-4 * np.abs(r[:, :, 1:3, 0]).max()
    # the gas has been set in motion
    assert tot1["ekin"] > 1e-3 * tot0["energy"]
