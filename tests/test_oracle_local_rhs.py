"""The oracle's right-hand side of single cells from their face
neighbourhoods (used for sampled parity at full mesh sizes) against its
whole-mesh right-hand side: same volume term, face fluxes and lifts (Sec. 2.2),
so the two agree to rounding; a wrong neighbour order, face side or sign would
show as an O(1) difference."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N,k", [(3, 1), (4, 2), (5, 3)])
@pytest.mark.parametrize("riemann", ["rusanov", "hllc"])
def test_cells_match_the_whole_mesh(N, k, riemann):
    u = I.random_state(N, k, seed=11 + k, v_rms=0.8)
    cfg = O.make_cfg(N, k, riemann=riemann)
    dt = 0.3 * (1 / N) / ((k + 1) * 4.0)
    full = O.rhs(cfg, u, None, dt)
    cells = np.arange(N ** 3)
    got = O.rhs_cells(cfg, u, cells, dt_pimax=dt)
    assert rel(got, full) < 1e-13


def test_forced_sample_with_global_mean():
    N, k = 5, 2
    u = I.random_state(N, k, seed=3, v_rms=0.5)
    a = I.random_state(N, k, seed=4, v_rms=0.5)[:, 1:, :].copy()
    cfg = O.make_cfg(N, k)
    dt = 1e-3
    full = O.rhs(cfg, u, a, dt)
    cells = np.array([0, 7, N ** 3 - 1, 2 * N * N + N + 3])
    got = O.rhs_cells(cfg, u, cells, ahat=a, abar=O.forcing_mean(cfg, u, a), dt_pimax=dt)
    assert rel(got, full[cells]) < 1e-13
    # without the global mean the momentum sources differ: the mean matters
    bad = O.rhs_cells(cfg, u, cells, ahat=a, abar=None, dt_pimax=dt)
    assert rel(bad, full[cells]) > 1e-6


def test_per_cell_coefficient():
    N, k = 4, 3
    u = I.random_state(N, k, seed=8, v_rms=0.8)
    nu = np.random.default_rng(1).uniform(0.0, 0.02, N ** 3)
    cfg = O.make_cfg(N, k)
    dt = 2e-3
    full = O.rhs_nu(cfg, u, nu, None, dt)
    cells = np.array([1, 5, 22, 63])
    got = O.rhs_cells(cfg, u, cells, dt_pimax=dt, nu_cell=nu[cells])
    assert rel(got, full[cells]) < 1e-13


def test_neighbourhood_is_periodic():
    nb = O.neighbourhood(4, [0, 63])
    assert list(nb[0]) == [0, 3, 1, 12, 4, 48, 16]
    assert list(nb[1]) == [63, 62, 60, 59, 51, 47, 15]


def test_tiled_state_gathers_from_the_base_mesh():
    # a 2^3 tiling of a 3^3 state is a 6^3 state; the RHS of its cells equals
    # the whole-mesh RHS of the tiled array
    k, n = 2, 3
    base = I.random_state(n, k, seed=21, v_rms=0.6)
    b = base.shape[-1]
    tiled = np.tile(base.reshape(n, n, n, 4, b), (2, 2, 2, 1, 1)).reshape(-1, 4, b)
    cfg = O.make_cfg(2 * n, k)
    full = O.rhs(cfg, tiled, None, 1e-3)
    cells = np.array([0, 5, 17, 100, 215])
    got = O.rhs_cells(cfg, base, cells, dt_pimax=1e-3, base_N=n)
    assert rel(got, full[cells]) < 1e-13
