"""Pins of the oracle's boundaries of the adiabatic system (outflow, reflective
and inflow faces along an axis; the paper's Shu-Osher and implosion problems,
Sec. 3.1, run between such faces).

A reflective wall is the mirror plane of a periodic problem of twice the
length: on a state that depends on x alone, the right-hand side between
walls equals that of the periodic box of twice the cells holding the state and
its mirror image (x -> -x, v_x -> -v_x), scaled by the ratio of the cell sizes.
Uniform flows stay put between outflow faces and behind an inflow of their own
state; walls conserve mass and energy exactly.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I

G = 1.4


def one_d_state(N, k, seed):
    """Coefficients [N^3][5][b] of a state that depends on x alone: the x-modes
    of random cells (i, 0, 0), copied along y and z."""
    u = I.random_energy_state(N, k, seed=seed, v_rms=0.3, p_mean=5.0, gamma=G)
    deg = I.mode_degrees(k)
    xonly = (deg[:, 1] == 0) & (deg[:, 2] == 0)
    out = np.zeros_like(u)
    for iz in range(N):
        for iy in range(N):
            for ix in range(N):
                src = ix                                   # cell (ix, 0, 0)
                out[(iz * N + iy) * N + ix] = u[src] * xonly[None, :]
    return out


def mirrored(u, N, k):
    """The same state on the (2N)^3 box of twice the length: x in [0, 1) as
    given, x in [1, 2) its mirror image (modes of odd x-degree and v_x flip)."""
    deg = I.mode_degrees(k)
    par = (-1.0) ** deg[:, 0]
    M = 2 * N
    out = np.zeros((M ** 3, 5, u.shape[2]))
    for iz in range(M):
        for iy in range(M):
            for ix in range(M):
                src = u[ix if ix < N else 2 * N - 1 - ix]          # 1D in x: any (iy, iz) of u
                if ix >= N:
                    src = src * par[None, :]
                    src = src.copy()
                    src[1] = -src[1]
                out[(iz * M + iy) * M + ix] = src
    return out


@pytest.mark.parametrize("k,riemann", [(1, "rusanov"), (2, "hllc")])
def test_reflective_walls_are_mirror_planes(k, riemann):
    N = 4
    u = one_d_state(N, k, seed=11 + k)
    walls = O.make_cfg(N, k, riemann=riemann, bc=("reflect", "periodic", "periodic"))
    r = O.adi_rhs(walls, G, u, 0.0)
    big = mirrored(u, N, k)
    rb = O.adi_rhs(O.make_cfg(2 * N, k, riemann=riemann), G, big, 0.0)
    assert np.isfinite(r).all() and np.isfinite(rb).all()
    # cells (ix, 0, 0): the doubled box has h/2, so its right-hand side is twice as large
    for ix in range(N):
        np.testing.assert_allclose(r[ix], 0.5 * rb[ix], rtol=1e-11, atol=1e-11)
    # with periodic faces the same state gives another right-hand side at the ends
    rp = O.adi_rhs(O.make_cfg(N, k, riemann=riemann), G, u, 0.0)
    assert np.abs(rp[0] - r[0]).max() > 1e-3


def test_walls_conserve_mass_and_energy():
    N, k = 4, 2
    u = I.random_energy_state(N, k, seed=5, v_rms=0.3, p_mean=5.0, gamma=G)
    cfg = O.make_cfg(N, k, bc=("reflect", "reflect", "reflect"))
    r = O.adi_rhs(cfg, G, u, 0.0)
    assert np.isfinite(r).all()
    for var in (0, 4):
        tot = r[:, var, 0].sum()
        assert abs(tot) < 1e-11 * np.abs(r[:, var, 0]).sum(), (var, tot)


@pytest.mark.parametrize("bc", ["outflow", "inflow"])
def test_uniform_flow_stays_put(bc):
    N, k = 4, 2
    rho, v, p = 1.3, np.array([2.1, -0.4, 0.7]), 0.9
    u = np.zeros((N ** 3, 5, O.nmodes(k)))
    u[:, 0, 0] = rho
    u[:, 1:4, 0] = rho * v
    u[:, 4, 0] = p / (G - 1) + 0.5 * rho * v @ v
    cfg = O.make_cfg(N, k, bc=(bc, "outflow", bc), inflow=(rho, *v, p))
    r = O.adi_rhs(cfg, G, u, 0.0)
    assert np.abs(r).max() < 1e-12


@pytest.mark.parametrize("riemann", ["rusanov", "hllc"])
def test_inflow_face_sees_the_prescribed_state(riemann):
    # a supersonic uniform inflow into a gas at rest: the first cell's mean
    # right-hand side is the flux difference F*(inflow, rest) - F(rest) over h
    N, k = 4, 1
    W_in = np.array([3.857143, 2.629369, 0.0, 0.0, 10.33333])
    u = np.zeros((N ** 3, 5, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    u[:, 4, 0] = 1.0 / (G - 1)
    cfg = O.make_cfg(N, k, riemann=riemann, bc=("inflow", "periodic", "periodic"), inflow=tuple(W_in))
    r = O.adi_rhs(cfg, G, u, 0.0)
    W_rest = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    flux = O.adi_rusanov if riemann == "rusanov" else O.adi_hllc
    F_in = flux(G, 0, W_in, W_rest)
    F_rest = flux(G, 0, W_rest, W_rest)
    h = 1.0 / N
    first = [(iz * N + iy) * N for iz in range(N) for iy in range(N)]
    for c in first:
        np.testing.assert_allclose(r[c, :, 0], (F_in - F_rest) / h, rtol=1e-12, atol=1e-12)
    # the cells behind it are untouched
    assert np.abs(r[[c + 1 for c in first]]).max() < 1e-12
