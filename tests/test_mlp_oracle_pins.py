"""Pins of the FP64 MLP reference and of the learned-sensor features/labels.

The network code is checked against central finite differences of its own
loss (independent of the hand-written backward pass), GELU's closed-form
values, Adam's known first step, and a regression problem whose optimum is
known; the sensor labels against the closed form of the viscous pressure on a
state with a known velocity divergence."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I


def test_gelu_values():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert M.gelu_prime(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    # gelu(z) -> z for large z, -> 0 for very negative z
    assert M.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-15)
    assert abs(M.gelu(np.array([-10.0]))[0]) < 1e-20
    # gelu(1) = Phi(1) = 0.841344746...
    assert M.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-14)
    # derivative by central differences
    z = np.linspace(-3, 3, 13)
    e = 1e-6
    fd = (M.gelu(z + e) - M.gelu(z - e)) / (2 * e)
    assert np.abs(fd - M.gelu_prime(z)).max() < 1e-8


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    D = 8
    th = M.init_params(D, seed=1, Hh=M.H)
    X = rng.normal(size=(32, D))
    y = rng.normal(size=32)
    loss, g = M.loss_and_grad(th, X, y)
    idx = rng.choice(th.size, 200, replace=False)
    eps = 1e-6
    for i in idx:
        tp = th.copy()
        tm = th.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (M.loss_and_grad(tp, X, y)[0] - M.loss_and_grad(tm, X, y)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert loss == pytest.approx(np.mean((M.forward(th, X) - y) ** 2), rel=1e-14)


def test_adam_first_step_is_lr_times_sign():
    th = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -1e-3, 7.0])
    opt = M.Adam(3, lr=0.01)
    opt.step(th, g)
    assert np.allclose(th, [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], atol=1e-9)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(3)
    D = 4
    X = rng.uniform(-1, 1, size=(2048, D))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    th = M.init_params(D, seed=2)
    hist = M.train(th, X, y, epochs=60, batch=256, lr=3e-3)
    assert hist[-1] < 0.02 * hist[0] and hist[-1] < 2e-3


def test_sensor_labels_closed_form():
    # rho = 1, v_x = -c (x - x_c): div v = -c at every point, so every cell's
    # nu = alpha (h/p)^2 c + beta cs (h/p), label log(nu/(cs h/p)); |v|hat is
    # the projection of c h/2 |xi_x|
    N, k, c = 4, 2, 6.0
    cfg = O.make_cfg(N, k, alpha=2.0, beta=0.2)
    b = O.nmodes(k)
    ml = [tuple(r) for r in O.mode_list(k)]
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, 0] = 1.0
    h = 1.0 / N
    u[:, 1, ml.index((1, 0, 0))] = -c * h / 2 / math.sqrt(3)
    x, y = O.av_features(cfg, u, 0.0)
    hp = h / (k + 1)
    nu = 2.0 * hp * hp * c + 0.2 * hp
    assert np.allclose(y, math.log(nu / hp), rtol=0, atol=1e-13)
    assert np.allclose(x[:, 0], 1.0) and np.allclose(x[:, 1:b], 0.0)
    # |v| = c h/2 |xi|; 3-point Gauss projection of |xi| onto Pn_0: (w_a |xi_a|)/2 = (5/9) sqrt(3/5)
    assert np.allclose(x[:, b], c * h / 2 * (5.0 / 9.0) * math.sqrt(0.6), atol=1e-14)
    # expansion: no compressive point, label at the floor max(beta, 0.05)
    u[:, 1, ml.index((1, 0, 0))] *= -1
    _, y2 = O.av_features(cfg, u, 0.0)
    assert np.allclose(y2, math.log(0.2))
    _, y3 = O.av_features(O.make_cfg(N, k, beta=0.0), u, 0.0)
    assert np.allclose(y3, math.log(0.05))


def pnorm(m, x):
    c = np.zeros(m + 1)
    c[m] = 1.0
    return math.sqrt(2 * m + 1) * npleg.legval(x, c)


@pytest.mark.parametrize("e", [4.0, 9.0])
def test_sensor_label_is_the_weighted_mean_over_compressive_points(e):
    # rho = 1, v_x(xi) with dv/dx = -c + e xi^2 (xi the cell's reference x):
    # div v varies over the Gauss points (and changes sign for e > c); the
    # label averages Pi/(rho |div v|) with the Gauss weights over the
    # compressive points only (the y, z weights cancel in the ratio)
    N, k, c = 4, 3, 6.0
    cfg = O.make_cfg(N, k, alpha=2.0, beta=0.2)
    b = O.nmodes(k)
    ml = [tuple(r) for r in O.mode_list(k)]
    h = 1.0 / N
    hp = h / (k + 1)
    # v(xi) = (h/2) (-c xi + e xi^3 / 3), projected on Pn_m by a 10-point Gauss rule
    t, w = npleg.leggauss(10)
    v = (h / 2) * (-c * t + e * t ** 3 / 3)
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, 0] = 1.0
    for m in range(k + 1):
        u[:, 1, ml.index((m, 0, 0))] = 0.5 * np.sum(w * v * pnorm(m, t))
    _, y = O.av_features(cfg, u, 0.0)
    xa, wa = npleg.leggauss(k + 1)
    D = -c + e * xa ** 2
    comp = D < 0
    nu_a = 2.0 * hp * hp * np.abs(D) + 0.2 * hp
    nu = np.sum(wa[comp] * nu_a[comp]) / np.sum(wa[comp])
    assert comp.any() and (e < c) == comp.all()
    assert np.allclose(y, math.log(max(nu, 0.2 * hp) / hp), rtol=0, atol=1e-12)
    if comp.all():
        # neither the maximum nor the unweighted mean (for e > c the two
        # compressive points share one value)
        assert abs(math.log(nu_a[comp].max() / hp) - y[0]) > 1e-3
        assert abs(math.log(nu_a[comp].mean() / hp) - y[0]) > 1e-4


def test_rhs_with_cell_coefficient_equals_vnr_when_nu_matches():
    # on the sawtooth state div v is constant, so nu = Pi/(rho |D|) per cell
    # reproduces the vNR right-hand side exactly
    N, k, c = 4, 2, 6.0
    cfg = O.make_cfg(N, k)
    b = O.nmodes(k)
    ml = [tuple(r) for r in O.mode_list(k)]
    u = I.uniform_state(N, k)
    u[:, 1, ml.index((1, 0, 0))] = -c * (1 / N) / 2 / math.sqrt(3)
    hp = (1 / N) / (k + 1)
    nu = np.full(N ** 3, 2.0 * hp * hp * c + 0.2 * hp)
    r1 = O.rhs(cfg, u, None, 0.0)
    r2 = O.rhs_nu(cfg, u, nu, None, 0.0)
    assert np.abs(r1 - r2).max() < 1e-11 * np.abs(r1).max()
    # and with nu = 0 the AV term vanishes
    r0 = O.rhs(O.make_cfg(N, k, av_mode=0), u, None, 0.0)
    assert np.abs(O.rhs_nu(cfg, u, np.zeros(N ** 3)) - r0).max() < 1e-12
