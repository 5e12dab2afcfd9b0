"""Pins of the oracle's diffusion operator div(eps grad u) with the
interface gradient from a recovered polynomial over the two neighbouring
cells (Sec. 2, diffusion across cell boundaries): recovery is exact for
polynomials it can represent, the operator is conservative, it converges to
the Laplacian of a smooth field, and a shear wave of the isothermal Euler
equations decays at the exact viscous rate."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I


def moments(f, shift, K):
    x, w = npleg.leggauss(16)
    out = []
    for a in range(K + 1):
        c = np.zeros(a + 1)
        c[a] = 1.0
        out.append(0.5 * np.sum(w * math.sqrt(2 * a + 1) * npleg.legval(x, c) * f(x + shift)))
    return out


@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_recovery_is_exact_for_degree_2K_plus_1(K):
    rng = np.random.default_rng(K)
    coef = rng.normal(size=2 * K + 2)
    f = lambda s: np.polynomial.polynomial.polyval(s, coef)  # noqa: E731
    d = O.recover_dn(K, moments(f, -1.0, K), moments(f, 1.0, K))
    assert abs(d - coef[1]) < 1e-12 * max(1.0, np.abs(coef).max())
    # an odd degree beyond 2K+1 is not reproduced (an added even power is:
    # its slope at the face is zero on both sides of the comparison)
    coef2 = np.concatenate([coef, [0.0, 1.0]])
    g = lambda s: np.polynomial.polynomial.polyval(s, coef2)  # noqa: E731
    d2 = O.recover_dn(K, moments(g, -1.0, K), moments(g, 1.0, K))
    assert abs(d2 - coef2[1]) > 1e-6


def test_diffusion_conserves_every_variable():
    N, k = 4, 2
    u = I.random_state(N, k, seed=3)
    r = O.diffusion_rhs(O.make_cfg(N, k, eps_diff=0.05), u)
    for v in range(4):
        assert abs(r[:, v, 0].sum()) < 1e-12 * np.abs(r[:, v, 0]).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_diffusion_of_a_sine_converges_to_the_laplacian(k):
    # rho = 1 + A sin(2 pi x): eps d^2/dx^2 gives -eps (2 pi)^2 A sin(2 pi x).
    # The cell means change by the difference of the recovered face
    # derivatives, accurate to O(h^(2k+1)) (the recovery reproduces degree
    # 2k+1): their error falls at least as h^2 (k = 1) and faster for k > 1.
    # (The highest modes of a DG right-hand side carry an O(h) consistency
    # error; the evolved solution converges anyway, see the shear wave test.)
    A, eps = 0.1, 0.01
    errs = []
    for N in (4, 8):
        b = O.nmodes(k)
        s = I.fourier_coeffs(N, k, (1, 0, 0)).imag
        u = np.zeros((N ** 3, 4, b))
        u[:, 0, 0] = 1.0
        u[:, 0, :] += A * s
        r = O.diffusion_rhs(O.make_cfg(N, k, eps_diff=eps), u)
        ref = -eps * (2 * np.pi) ** 2 * A * s
        errs.append(np.linalg.norm(r[:, 0, 0] - ref[:, 0]) / np.linalg.norm(ref[:, 0]))
        assert np.abs(r[:, 1:]).max() < 1e-14
    rate = math.log2(errs[0] / errs[1])
    assert rate > (1.9 if k == 1 else 3.5), (errs, rate)


@pytest.mark.parametrize("k,tol", [(1, 2e-2), (2, 1e-2), (3, 2e-4)])
def test_shear_wave_decays_at_the_viscous_rate(k, tol):
    # rho = 1, v_y = A sin(2 pi x): a steady solution of isothermal Euler; with
    # div(eps grad u) the momentum decays as exp(-eps (2 pi)^2 t).  HLLC (no
    # tangential flux for v_x = 0), no viscous pressure; eps large enough that
    # the diffusive time-step limit binds (stability of the explicit scheme)
    N, A, eps = 8, 0.05, 0.2
    b = O.nmodes(k)
    s = I.fourier_coeffs(N, k, (1, 0, 0)).imag
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, 0] = 1.0
    u[:, 2, :] = A * s
    cfg = O.make_cfg(N, k, av_mode=0, riemann="hllc", eps_diff=eps)
    hp = (1.0 / N) / (k + 1)
    assert abs(O.dt(cfg, u) - 0.3 * hp * hp / (2 * eps)) < 1e-15
    rc, t, _, _ = O.run(cfg, u, 60)
    assert rc == 0
    amp = np.sum(u[:, 2, :] * s) / np.sum(s * s)
    assert abs(amp / (A * math.exp(-eps * (2 * np.pi) ** 2 * t)) - 1) < tol, (amp, t)
    assert np.abs(u[:, 0, 1:]).max() < 1e-12 and np.abs(u[:, 1, :]).max() < 1e-12
