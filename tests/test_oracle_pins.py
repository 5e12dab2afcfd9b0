"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
textbook special cases (numpy's Gauss-Legendre / Legendre routines), exact
invariants of the weak form, the exact translation of a linear sound wave, the
stability polynomial of the SSP Runge-Kutta schemes, and published test
vectors.  A plausible mistake anywhere in the oracle (a dropped term, a sign,
an index, a transposed operand, a wrong normalisation) fails one of them.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# independent evaluation helpers (numpy's Legendre series, not the oracle)
# --------------------------------------------------------------------------

def pnorm(m, x):
    c = np.zeros(m + 1)
    c[m] = 1.0
    return math.sqrt(2 * m + 1) * npleg.legval(x, c)


def eval_cell(coef, k, xi):
    """coef [b] at reference points xi [P,3] with numpy's Legendre series."""
    ijl = I.mode_degrees(k)
    out = np.zeros(len(xi))
    for l, (i, j, m) in enumerate(ijl):
        out += coef[l] * pnorm(i, xi[:, 0]) * pnorm(j, xi[:, 1]) * pnorm(m, xi[:, 2])
    return out


def check_points(k):
    """volume Gauss points and the face Gauss points of all six faces."""
    g, _ = npleg.leggauss(k + 1)
    A, B, C = np.meshgrid(g, g, g, indexing="ij")
    vol = np.stack([A.ravel(), B.ravel(), C.ravel()], 1)
    T1, T2 = np.meshgrid(g, g, indexing="ij")
    faces = []
    for d in range(3):
        for s in (-1.0, 1.0):
            p = np.zeros((T1.size, 3))
            t = [e for e in range(3) if e != d]
            p[:, d] = s
            p[:, t[0]] = T1.ravel()
            p[:, t[1]] = T2.ravel()
            faces.append(p)
    return np.concatenate([vol] + faces)


def l1_vs_exact(u, N, k, fn, nq=None):
    """(1/V) int |rho_h - rho_exact| by (k+4)-point numpy Gauss per axis."""
    nq = nq or k + 4
    g, w = npleg.leggauss(nq)
    A, B, C = np.meshgrid(g, g, g, indexing="ij")
    xi = np.stack([A.ravel(), B.ravel(), C.ravel()], 1)
    W = np.einsum("a,b,c->abc", w, w, w).ravel() / 8.0
    h = 1.0 / N
    ijl = I.mode_degrees(k)
    Phi = np.stack([pnorm(i, xi[:, 0]) * pnorm(j, xi[:, 1]) * pnorm(m, xi[:, 2]) for (i, j, m) in ijl], 1)
    rho = u[:, 0, :] @ Phi.T                  # [cells][points]
    iz, iy, ix = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    xc = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) + 0.5
    X = (xc[:, None, :] + 0.5 * xi[None, :, :]) * h
    return float((np.abs(rho - fn(X)) * W[None, :]).sum() * h ** 3)


# --------------------------------------------------------------------------
# 1D building blocks
# --------------------------------------------------------------------------

def test_gauss_closed_forms_and_exactness():
    x, w = O.gauss(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15, rtol=0)
    assert np.allclose(w, [1, 1], atol=1e-15, rtol=0)
    x, w = O.gauss(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15, rtol=0)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15, rtol=0)
    x, w = O.gauss(4)
    a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
    b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    assert np.allclose(x, [-b, -a, a, b], atol=1e-15, rtol=0)
    wa, wb = (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36
    assert np.allclose(w, [wb, wa, wa, wb], atol=1e-15, rtol=0)
    for n in range(1, 9):
        x, w = O.gauss(n)
        xr, wr = npleg.leggauss(n)
        assert np.allclose(x, xr, atol=2e-15, rtol=0) and np.allclose(w, wr, atol=2e-15, rtol=0)
        assert abs(w.sum() - 2) < 1e-14
        for p in range(2 * n):  # exact up to degree 2n-1
            exact = 0.0 if p % 2 else 2.0 / (p + 1)
            assert abs((w * x ** p).sum() - exact) < 1e-14
        assert abs((w * x ** (2 * n)).sum() - 2.0 / (2 * n + 1)) > 1e-6  # and not beyond


def test_legendre_values_and_derivatives():
    xs = np.linspace(-1, 1, 11)
    for x in xs:
        assert abs(O.legendre(2, x) - (3 * x * x - 1) / 2) < 1e-15
        assert abs(O.legendre(3, x) - (5 * x ** 3 - 3 * x) / 2) < 1e-15
        assert abs(O.legendre(4, x) - (35 * x ** 4 - 30 * x ** 2 + 3) / 8) < 1e-15
        assert abs(O.legendre_deriv(2, x) - 3 * x) < 1e-15
        assert abs(O.legendre_deriv(3, x) - (15 * x * x - 3) / 2) < 1e-14
        assert abs(O.legendre_deriv(4, x) - (140 * x ** 3 - 60 * x) / 8) < 1e-13
        for m in range(9):
            c = np.zeros(m + 1)
            c[m] = 1
            assert abs(O.legendre(m, x) - npleg.legval(x, c)) < 1e-14
            assert abs(O.legendre_deriv(m, x) - npleg.legval(x, npleg.legder(c))) < 1e-12
    for m in range(9):
        assert O.legendre(m, 1.0) == pytest.approx(1.0, abs=1e-15)
        assert O.legendre(m, -1.0) == pytest.approx((-1) ** m, abs=1e-15)


def test_mode_list_order():
    assert O.mode_list(1).tolist() == [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    assert O.mode_list(2)[4:].tolist() == [[2, 0, 0], [1, 1, 0], [1, 0, 1], [0, 2, 0], [0, 1, 1], [0, 0, 2]]
    for k in range(1, 5):
        ml = O.mode_list(k)
        assert len(ml) == O.nmodes(k) == (k + 1) * (k + 2) * (k + 3) // 6
        assert (ml == I.mode_degrees(k)).all()
        assert len({tuple(r) for r in ml}) == len(ml) and ml.sum(1).max() == k


# --------------------------------------------------------------------------
# projection (Sec. 3.2) and orthonormality (Sec. 2.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3])
def test_projection_is_identity_for_polynomial_velocity(k):
    # rho = 1: v = m is a degree-k polynomial, so the projection returns it
    # exactly iff the basis is orthonormal and the quadrature exact (Sec. 2.2).
    N = 3
    u = I.random_state(N, k, seed=11)
    u[:, 0, :] = 0.0
    u[:, 0, 0] = 1.0
    vh = O.project_velocity(O.make_cfg(N, k), u)
    assert np.abs(vh - u[:, 1:, :]).max() < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3])
def test_projection_of_constant_velocity(k):
    # m = c rho with any positive rho: v = c, so vhat = c delta_l0.
    N = 3
    u = I.random_state(N, k, seed=12)
    c = np.array([0.3, -1.7, 2.5])
    for i in range(3):
        u[:, 1 + i, :] = c[i] * u[:, 0, :]
    vh = O.project_velocity(O.make_cfg(N, k), u)
    assert np.abs(vh[:, :, 0] - c[None, :]).max() < 1e-13
    assert np.abs(vh[:, :, 1:]).max() < 1e-13


# --------------------------------------------------------------------------
# weak form invariants (Sec. 2.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3])
def test_uniform_state_is_steady(k):
    cfg = O.make_cfg(4, k)
    u = I.uniform_state(4, k, rho=1.3, v=(0.2, -0.1, 0.05))
    r = O.rhs(cfg, u, None, 1e-3)
    assert np.abs(r).max() < 1e-13


@pytest.mark.parametrize("k", [1, 2, 3])
def test_conservation_of_mass_and_momentum(k):
    N = 4
    cfg = O.make_cfg(N, k)
    u = I.random_state(N, k, seed=5)
    fo = O.Forcing(mach=2.0, zeta=0.5, seed=3)
    ahat = O.forcing_project(cfg, fo.kvec(), fo.amplitudes())
    for a in (None, ahat):
        r = O.rhs(cfg, u, a, 1e-3)
        scale = np.abs(r[:, :, 0]).max()
        assert scale > 1.0
        tot = r[:, :, 0].sum(axis=0)
        assert np.abs(tot).max() < 1e-12 * scale * N ** 3


def test_rusanov_identities():
    rng = np.random.default_rng(0)
    cs = 1.3
    for _ in range(20):
        WL = np.array([rng.uniform(0.2, 3), *rng.normal(size=3)])
        WR = np.array([rng.uniform(0.2, 3), *rng.normal(size=3)])
        for d in range(3):
            # consistency: F*(U,U) = physical flux
            F = O.rusanov(cs, d, WL, WL)
            phys = np.array([WL[0] * WL[1 + d]] + [WL[0] * WL[1 + i] * WL[1 + d] + (cs * cs * WL[0] if i == d else 0)
                                                   for i in range(3)])
            assert np.allclose(F, phys, rtol=1e-14, atol=1e-14)
            # mirror antisymmetry: reflecting the problem along d flips the flux
            M = np.ones(4)
            M[1 + d] = -1
            Fm = O.rusanov(cs, d, WR * M, WL * M)
            assert np.allclose(Fm * M, -O.rusanov(cs, d, WL, WR), rtol=1e-13, atol=1e-13)
            # dissipation: lambda = max|v_d| + cs multiplies the jump
            F1 = O.rusanov(cs, d, WL, WR)
            lam = max(abs(WL[1 + d]), abs(WR[1 + d])) + cs
            UL = np.concatenate([[WL[0]], WL[0] * WL[1:]])
            UR = np.concatenate([[WR[0]], WR[0] * WR[1:]])
            avg = 0.5 * (O.rusanov(cs, d, WL, WL) + O.rusanov(cs, d, WR, WR))
            assert np.allclose(F1, avg - 0.5 * lam * (UR - UL), rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# von Neumann-Richtmyer viscosity (Sec. 3.1)
# --------------------------------------------------------------------------

def test_vnr_values():
    N, k = 8, 2
    cfg = O.make_cfg(N, k, alpha=2.0, beta=0.2, cs=1.5)
    hp = (1 / N) / (k + 1)
    for d in (0.0, 0.5, 3.0):
        assert O.vnr(cfg, 1.7, d, 1e-3) == 0.0
    rho, D = 1.7, -3.0
    expect = 2.0 * rho * hp ** 2 * 9.0 + 0.2 * rho * 1.5 * hp * 3.0
    assert O.vnr(cfg, rho, D, 0.0) == pytest.approx(expect, rel=1e-15)
    # cap Pi_max = rho (h/p)^2 |D| / (2 dt) becomes active for a large dt*|D|
    dt = 0.5 * hp ** 2 * 3.0 * rho / expect * 2.0
    assert O.vnr(cfg, rho, D, dt) == pytest.approx(0.5 * rho * hp ** 2 * 3.0 / dt, rel=1e-15)
    cfg0 = O.make_cfg(N, k, av_mode=0)
    assert O.vnr(cfg0, rho, D, 0.0) == 0.0


def _sawtooth(N, k, c, a=0.0):
    """rho = 1 + a xi_x, v_x = -c (h/2) xi_x inside every cell (div v = -c exactly)."""
    b = O.nmodes(k)
    ml = [tuple(r) for r in O.mode_list(k)]
    h = 1.0 / N
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, ml.index((0, 0, 0))] = 1.0
    u[:, 0, ml.index((1, 0, 0))] = a / math.sqrt(3)
    # m_x = -c h/2 (xi + a xi^2);  xi = Pn_1/sqrt3;  xi^2 = 1/3 + (2/3) P_2 = 1/3 + 2 Pn_2/(3 sqrt5)
    u[:, 1, ml.index((1, 0, 0))] = -c * h / 2 / math.sqrt(3)
    u[:, 1, ml.index((0, 0, 0))] = -c * h / 2 * a / 3
    if a != 0.0:
        u[:, 1, ml.index((2, 0, 0))] = -c * h / 2 * a * 2 / (3 * math.sqrt(5))
    return u


@pytest.mark.parametrize("k", [1, 2, 3])
def test_viscous_pressure_enters_volume_term_only(k):
    # rho = 1, v_x = -c (x - x_c): Pi is constant in the cell, so its only
    # effect on the weak form is (1/(4h)) sum_q w_q dphi/dxi_x Pi, whose closed
    # form for the mode (i,0,0) is Pi sqrt(2i+1) (1 - (-1)^i) / h.
    N, c = 4, 7.0
    h, hp = 1.0 / N, 1.0 / N / (k + 1)
    u = _sawtooth(N, k, c)
    cfg_on = O.make_cfg(N, k, alpha=2.0, beta=0.2)
    cfg_off = O.make_cfg(N, k, av_mode=0)
    Pi = 2.0 * hp ** 2 * c * c + 0.2 * hp * c
    ml = [tuple(r) for r in O.mode_list(k)]
    dR = O.rhs(cfg_on, u, None, 0.0) - O.rhs(cfg_off, u, None, 0.0)
    # Pi is isotropic: m_d receives the same term along its own axis d
    expect = np.zeros((4, O.nmodes(k)))
    for d in range(3):
        for i in range(1, k + 1):
            deg = [0, 0, 0]
            deg[d] = i
            expect[1 + d, ml.index(tuple(deg))] = Pi * math.sqrt(2 * i + 1) * (1 - (-1) ** i) / h
    assert np.abs(dR - expect[None]).max() < 1e-11 * Pi / h
    # the cap: with a large dt the limited Pi_max = rho (h/p)^2 c /(2 dt) is used
    dt = 1.0 * hp ** 2 * c / Pi
    dR2 = O.rhs(cfg_on, u, None, dt) - O.rhs(cfg_off, u, None, dt)
    Pmax = 0.5 * hp ** 2 * c / dt
    assert Pmax < Pi
    assert dR2[0, 1, ml.index((1, 0, 0))] == pytest.approx(Pmax * 2 * math.sqrt(3) / h, rel=1e-11)
    # expansion (c < 0): no viscous pressure
    dR3 = O.rhs(cfg_on, _sawtooth(N, k, -c), None, 0.0) - O.rhs(cfg_off, _sawtooth(N, k, -c), None, 0.0)
    assert np.abs(dR3).max() < 1e-12


@pytest.mark.parametrize("k", [2, 3])
def test_divergence_uses_quotient_rule(k):
    # rho = 1 + a xi_x with v linear: div v = -c exactly, and Pi ~ rho_q.
    # (1/(4h)) sum_q w_q dphi_(2,0,0)/dxi_x Pi_1 (1 + a xi) = 2 sqrt5 a Pi_1 / h,
    # (1,0,0) keeps 2 sqrt3 Pi_1 / h.  div(m)/rho alone would give a different div v.
    N, c, a = 4, 5.0, 0.4
    h, hp = 1.0 / N, 1.0 / N / (k + 1)
    u = _sawtooth(N, k, c, a)
    Pi1 = 2.0 * hp ** 2 * c * c + 0.2 * hp * c
    ml = [tuple(r) for r in O.mode_list(k)]
    dR = O.rhs(O.make_cfg(N, k), u, None, 0.0) - O.rhs(O.make_cfg(N, k, av_mode=0), u, None, 0.0)
    assert dR[0, 1, ml.index((1, 0, 0))] == pytest.approx(2 * math.sqrt(3) * Pi1 / h, rel=1e-11)
    assert dR[0, 1, ml.index((2, 0, 0))] == pytest.approx(2 * math.sqrt(5) * a * Pi1 / h, rel=1e-11)


# --------------------------------------------------------------------------
# time integration (Sec. 7)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k,stages", [(1, 2), (2, 3), (1, 3)])
def test_ssp_rk_stability_polynomial(k, stages):
    # Linearised about rest, one step is R(dt A) w with R(z) = 1 + z + z^2/2
    # (SSP-RK2) or 1 + z + z^2/2 + z^3/6 (SSP-RK3), A the linearised RHS.
    N = 4
    cfg = O.make_cfg(N, k, av_mode=0, rk_stages=stages)
    u0 = I.uniform_state(N, k)
    w = I.random_state(N, k, seed=21)
    w[:, 0, 0] -= w[:, 0, 0].mean()
    # the max|v_n| of the Rusanov flux is only Lipschitz at rest: the central
    # difference keeps an O(eps) remainder, hence the small eps
    eps = 1e-6

    def A(v):
        s = np.abs(v).max()
        return (O.rhs(cfg, u0 + eps * v / s) - O.rhs(cfg, u0 - eps * v / s)) / (2 * eps) * s

    dt = 0.3 * (1 / N) / ((k + 1) * 3)
    up, um = u0 + eps * w, u0 - eps * w
    O.step(cfg, up, None, dt)
    O.step(cfg, um, None, dt)
    S = (up - um) / (2 * eps)
    Aw = A(w)
    AAw = A(Aw)
    R = w + dt * Aw + dt ** 2 / 2 * AAw
    if stages == 3:
        R = R + dt ** 3 / 6 * A(AAw)
    assert np.abs(S - R).max() < 1e-6 * np.abs(w).max()
    # the cubic term is large enough that a wrong stage weight would show
    if stages == 3:
        assert np.abs(dt ** 3 / 6 * A(AAw)).max() > 1e-3 * np.abs(w).max()


def test_cfl_dt_closed_form():
    for k in (1, 2, 3):
        N = 4
        u = I.uniform_state(N, k, rho=0.7, v=(0.3, -0.4, 0.1))
        cfg = O.make_cfg(N, k, cs=2.0, cfl=0.3)
        expect = 0.3 * (1 / N) / ((k + 1) * (0.3 + 0.4 + 0.1 + 3 * 2.0))
        assert O.dt(cfg, u) == pytest.approx(expect, rel=1e-14)


# --------------------------------------------------------------------------
# order of accuracy on a linear sound wave (Sec. 2.2: L1 ~ h^(k+1))
# --------------------------------------------------------------------------

def _wave_error(N, k, nsteps, kvec=(1, 0, 0), v0=(0, 0, 0), cfl=0.3):
    eps = 1e-6
    cfg = O.make_cfg(N, k, av_mode=0, cfl=cfl)
    u = I.sound_wave(N, k, eps=eps, kvec=kvec, v0=v0)
    rc, t, _, _ = O.run(cfg, u, nsteps)
    assert rc == 0
    kv = np.array(kvec, float)
    kn = np.linalg.norm(kv)
    w = 2 * np.pi * kn * (1.0 + (kv / kn) @ np.array(v0, float))
    err = l1_vs_exact(u, N, k, lambda X: 1 + eps * np.sin(2 * np.pi * X @ kv - w * t))
    return err / eps


@pytest.mark.parametrize("k", [1, 2])
def test_sound_wave_convergence(k):
    e1 = _wave_error(8, k, 12)
    e2 = _wave_error(16, k, 24)
    rate = math.log2(e1 / e2)
    assert rate > k + 0.75, (e1, e2, rate)


@pytest.mark.slow
def test_sound_wave_convergence_k3():
    # RK3 is one order short of the space order at k=3; a small CFL keeps the
    # time error below the spatial one.
    e1 = _wave_error(4, 3, 20, cfl=0.05)
    e2 = _wave_error(8, 3, 40, cfl=0.05)
    assert math.log2(e1 / e2) > 3.6


def test_sound_wave_galilean_diagonal():
    e1 = _wave_error(8, 2, 16, kvec=(1, 1, 0), v0=(0.3, -0.2, 0.1))
    e2 = _wave_error(16, 2, 32, kvec=(1, 1, 0), v0=(0.3, -0.2, 0.1))
    assert math.log2(e1 / e2) > 2.7


# --------------------------------------------------------------------------
# driving (Sec. 4.2)
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        ref = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    assert O.splitmix64(0, 3) == ref


def test_ou_mode_set_and_projection():
    fo = O.Forcing(mach=3.0, zeta=1.0, seed=1)
    kv = fo.kvec()
    assert fo.nmodes == 61 == len(kv)
    r2 = (kv ** 2).sum(1)
    assert r2.min() == 1 and r2.max() == 9
    full = {tuple(v) for v in kv} | {tuple(-v) for v in kv}
    assert len(full) == 122
    amp = fo.amplitudes()
    # purely solenoidal: k . a = 0
    assert np.abs(np.einsum("mi,mir->mr", kv, amp)).max() < 1e-14
    fo0 = O.Forcing(mach=3.0, zeta=0.0, seed=1)
    amp0 = fo0.amplitudes()
    # purely compressive: k x a = 0
    assert np.abs(np.cross(kv[:, :, None], amp0, axis=1)).max() < 1e-14


def test_ou_process_statistics():
    mach, zeta = 2.0, 0.5
    fo = O.Forcing(mach=mach, zeta=zeta, seed=9)
    tc = 1.0 / (2 * mach)
    f = math.exp(-0.01)
    s = (2 * mach ** 2) / math.sqrt(4 * 61 * (2 * zeta ** 2 + (1 - zeta) ** 2))
    xs = [fo.x()]
    for _ in range(300):
        fo.advance()
        xs.append(fo.x())
    X = np.array(xs).reshape(len(xs), -1)
    z = (X[1:] - f * X[:-1]) / (s * math.sqrt(1 - f * f))
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    # lag-one correlation of the innovations vanishes
    assert abs((z[1:] * z[:-1]).mean()) < 4 / math.sqrt(n)
    # stationary start: Var x = s^2 over several seeds
    x0 = np.concatenate([O.Forcing(mach, zeta, seed=sd).x().ravel() for sd in range(20)])
    assert abs(x0.var() / s ** 2 - 1) < 4 * math.sqrt(2 / x0.size)
    assert fo.ou.tc == pytest.approx(tc) and fo.ou.dt_drive == pytest.approx(tc / 100)


@pytest.mark.parametrize("kvec", [(1, 0, 0), (1, 2, -2)])
def test_forcing_projection_matches_exact_coefficients(kvec):
    # single mode: a_y(x) = 2 Re(A e^{2 pi i k.x}); the Gauss projection equals
    # the exact L2 coefficients (spherical Bessel closed form) up to the
    # (k+1)-point quadrature error.
    N, k = 8, 3
    cfg = O.make_cfg(N, k)
    A = 0.3 - 0.7j
    amp = np.zeros((1, 3, 2))
    amp[0, 1] = [A.real, A.imag]
    ah = O.forcing_project(cfg, np.array([kvec]), amp)
    ex = 2 * (A * I.fourier_coeffs(N, k, kvec)).real
    assert np.abs(ah[:, 1, :] - ex).max() < 2e-4
    assert np.abs(ah[:, [0, 2], :]).max() == 0.0
    # and it converges with N at the quadrature's rate
    ah2 = O.forcing_project(O.make_cfg(2 * N, k), np.array([kvec]), amp)
    ex2 = 2 * (A * I.fourier_coeffs(2 * N, k, kvec)).real
    # highest mode: the n-point rule errs like h^(2n-k) = h^5 at k=3
    assert np.abs(ah2[:, 1, :] - ex2).max() < np.abs(ah[:, 1, :] - ex).max() / 20


def test_forcing_source_on_uniform_gas():
    # rho = 1, v = 0: all fluxes are constant, so the RHS of m is the forcing
    # coefficient minus the mean acceleration (zero for a pure Fourier mode).
    N, k = 4, 2
    cfg = O.make_cfg(N, k)
    fo = O.Forcing(mach=1.0, zeta=0.5, seed=4)
    ah = O.forcing_project(cfg, fo.kvec(), fo.amplitudes())
    r = O.rhs(cfg, I.uniform_state(N, k), ah, 1e-3)
    assert np.abs(r[:, 1:, :] - ah).max() < 1e-13 * np.abs(ah).max() * 10
    assert np.abs(r[:, 0, :]).max() < 1e-13


# --------------------------------------------------------------------------
# positivity (Sec. 3.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3])
def test_limiter_rescales_to_floor(k):
    N = 2
    cfg = O.make_cfg(N, k, rho_floor=1e-3)
    u = I.random_state(N, k, seed=3, rho_wiggle=0.5)
    ml = [tuple(r) for r in O.mode_list(k)]
    u[0, 0, ml.index((1, 0, 0))] = 0.9 * u[0, 0, 0]   # goes negative at xi_x = -1
    before = u.copy()
    pts = check_points(k)
    assert eval_cell(before[0, 0], k, pts).min() < 0
    st = O.limit(cfg, u)
    assert st == O.ORC_LIMITED
    assert np.array_equal(u[:, :, 0], before[:, :, 0])  # means untouched
    theta = u[0, 1, 1] / before[0, 1, 1]
    assert 0 < theta < 1
    assert np.allclose(u[0, :, 1:], theta * before[0, :, 1:], rtol=1e-14, atol=0)
    assert eval_cell(u[0, 0], k, pts).min() == pytest.approx(1e-3, abs=1e-14)
    assert np.array_equal(u[1:], before[1:])
    # a mean at the floor cannot be repaired
    u[1, 0, 0] = 5e-4
    assert O.limit(cfg, u) & O.ORC_FAIL


def test_failed_step_is_retried_then_reported():
    N, k = 2, 1
    cfg = O.make_cfg(N, k)
    u = I.uniform_state(N, k)
    # a negative cell mean: the inflow of one stage cannot lift it above the
    # floor for any dt, so every retry fails
    u[3, 0, 0] = -1.0
    before = u.copy()
    rc, t, _, _ = O.run(cfg, u, 1)
    assert rc == -1 and t == 0.0
    assert np.array_equal(u, before)


# --------------------------------------------------------------------------
# diagnostics and the L1 norm
# --------------------------------------------------------------------------

def test_diagnostics_of_uniform_flow():
    k = 2
    u = I.uniform_state(4, k, rho=2.0, v=(0.3, 0.0, -0.4))
    d = O.diagnostics(O.make_cfg(4, k, cs=0.5), u)
    assert d["mass"] == pytest.approx(2.0, rel=1e-14)
    assert d["mom_x"] == pytest.approx(0.6, rel=1e-14) and d["mom_z"] == pytest.approx(-0.8, rel=1e-14)
    assert d["ekin"] == pytest.approx(0.5 * 2.0 * 0.25, rel=1e-13)
    assert d["mach"] == pytest.approx(0.5 / 0.5, rel=1e-13)
    assert d["mach_rho"] == pytest.approx(1.0, rel=1e-13)
    assert d["rho_min"] == pytest.approx(2.0) and d["rho_max"] == pytest.approx(2.0)
    assert d["av_frac"] == 0.0 and d["max_speed"] == pytest.approx(0.7 + 1.5)


def test_l1_density_norm():
    k, N = 2, 4
    cfg = O.make_cfg(N, k)
    a = I.random_state(N, k, seed=1)
    b = a.copy()
    b[:, 0, 0] += 0.25
    assert O.l1_density(cfg, a, b) == pytest.approx(0.25, rel=1e-13)
    # a non-constant difference: the same (k+3)-point rule evaluated with numpy
    c = a.copy()
    c[:, 0, 1] += 0.1
    c[:, 0, 5] -= 0.05
    diff = np.zeros_like(a)
    diff[:, 0, 1] = 0.1
    diff[:, 0, 5] = -0.05
    want = l1_vs_exact(diff, N, k, lambda X: 0.0 * X[..., 0], nq=k + 3)
    assert O.l1_density(cfg, c, a) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("N", [3, 4])
def test_oracle_is_independent_of_the_thread_count(N):
    # the parallel loops (cells; interfaces in parity colours; fixed-block sums)
    # give the same bits for any number of threads, odd meshes included
    k = 2
    out = []
    for th in (1, 3):
        O.set_threads(th)
        u = I.random_state(N, k, seed=8, v_rms=0.6)
        rc, t, _, _ = O.run(O.make_cfg(N, k), u, 2, forcing=O.Forcing(mach=2.0, zeta=0.5, seed=1))
        assert rc == 0
        out.append((u, t))
    O.set_threads(os.cpu_count() or 1)
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
