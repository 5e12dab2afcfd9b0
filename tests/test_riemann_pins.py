"""Pins of the oracle's HLL and HLLC face fluxes (the paper's solver family,
Sec. 2) against facts of the isothermal Euler equations: consistency with the
physical flux, upwinding in supersonic flow, mirror symmetry, the exact
steady contact (shear) discontinuity that HLLC keeps and HLL smears, and the
exact solution of the isothermal Riemann problem that the full scheme must
converge to."""
import math

import numpy as np
import pytest

from oracle import oracle as O

SOLVERS = ("hll", "hllc")


def phys_flux(cs, d, W):
    return np.array([W[0] * W[1 + d]] + [W[0] * W[1 + i] * W[1 + d] + (cs * cs * W[0] if i == d else 0.0)
                                         for i in range(3)])


def cons(W):
    return np.concatenate([[W[0]], W[0] * W[1:]])


@pytest.mark.parametrize("solver", SOLVERS)
def test_consistency_and_mirror_symmetry(solver):
    rng = np.random.default_rng(11)
    cs = 0.9
    for _ in range(40):
        WL = np.array([rng.uniform(0.2, 3), *rng.normal(size=3)])
        WR = np.array([rng.uniform(0.2, 3), *rng.normal(size=3)])
        for d in range(3):
            assert np.allclose(O.riemann(solver, cs, d, WL, WL), phys_flux(cs, d, WL), rtol=1e-14, atol=1e-14)
            M = np.ones(4)
            M[1 + d] = -1.0
            Fm = O.riemann(solver, cs, d, WR * M, WL * M)
            assert np.allclose(Fm * M, -O.riemann(solver, cs, d, WL, WR), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("solver", SOLVERS)
def test_supersonic_upwinding(solver):
    # all signal speeds of one sign: the flux is the upwind physical flux
    cs = 1.0
    WL = np.array([1.3, 2.5, 0.4, -0.7])
    WR = np.array([0.6, 1.8, -0.2, 0.3])
    assert np.allclose(O.riemann(solver, cs, 0, WL, WR), phys_flux(cs, 0, WL), rtol=1e-15, atol=1e-15)
    WL2 = np.array([1.3, -2.5, 0.4, -0.7])
    WR2 = np.array([0.6, -1.8, -0.2, 0.3])
    assert np.allclose(O.riemann(solver, cs, 0, WL2, WR2), phys_flux(cs, 0, WR2), rtol=1e-15, atol=1e-15)


def test_hll_closed_form_and_hllc_shares_mass_and_normal_momentum():
    rng = np.random.default_rng(12)
    cs = 1.1
    for _ in range(40):
        WL = np.array([rng.uniform(0.2, 3), *rng.normal(scale=0.5, size=3)])
        WR = np.array([rng.uniform(0.2, 3), *rng.normal(scale=0.5, size=3)])
        d = int(rng.integers(3))
        SL = min(WL[1 + d], WR[1 + d]) - cs
        SR = max(WL[1 + d], WR[1 + d]) + cs
        assert SL < 0 < SR
        FL, FR = phys_flux(cs, d, WL), phys_flux(cs, d, WR)
        ref = (SR * FL - SL * FR + SL * SR * (cons(WR) - cons(WL))) / (SR - SL)
        F = O.riemann("hll", cs, d, WL, WR)
        assert np.allclose(F, ref, rtol=1e-13, atol=1e-14)
        G = O.riemann("hllc", cs, d, WL, WR)
        assert abs(G[0] - F[0]) < 1e-13 and abs(G[1 + d] - F[1 + d]) < 1e-13
        # tangential momentum leaves with the mass flux at the upwind tangential velocity
        rs = (SR * WR[0] - SL * WL[0] - (FR[0] - FL[0])) / (SR - SL)
        ms = (SR * cons(WR)[1 + d] - SL * cons(WL)[1 + d] - (FR[1 + d] - FL[1 + d])) / (SR - SL)
        Wup = WL if ms / rs >= 0 else WR
        for t in range(3):
            if t != d:
                assert abs(G[1 + t] - G[0] * Wup[1 + t]) < 1e-12


def test_steady_shear_layer_is_exact_for_hllc_only():
    # equal density and pressure, no normal velocity, a jump in the tangential
    # velocity: a steady contact.  HLLC returns its exact flux; HLL diffuses it.
    cs = 1.0
    WL = np.array([1.4, 0.0, 0.8, -0.3])
    WR = np.array([1.4, 0.0, -0.5, 0.6])
    exact = np.array([0.0, cs * cs * 1.4, 0.0, 0.0])
    assert np.allclose(O.riemann("hllc", cs, 0, WL, WR), exact, atol=1e-15)
    F = O.riemann("hll", cs, 0, WL, WR)
    assert abs(F[2]) > 0.1 and abs(F[3]) > 0.1
    # at the scheme level: a piecewise-constant shear layer is a steady state of
    # the HLLC scheme (right-hand side zero), not of the HLL scheme
    N, k = 4, 2
    b = O.nmodes(k)
    u = np.zeros((N ** 3, 4, b))
    ix = np.arange(N ** 3) % N
    u[:, 0, 0] = 1.4
    u[:, 2, 0] = np.where(ix < N // 2, 1.4 * 0.8, -1.4 * 0.5)
    u[:, 3, 0] = np.where(ix < N // 2, -1.4 * 0.3, 1.4 * 0.6)
    r_hllc = O.rhs(O.make_cfg(N, k, riemann="hllc"), u)
    r_hll = O.rhs(O.make_cfg(N, k, riemann="hll"), u)
    assert np.abs(r_hllc).max() < 1e-13
    assert np.abs(r_hll).max() > 1e-2


# --------------------------------------------------------------------------
# exact solution of the isothermal Riemann problem (test helper)
# --------------------------------------------------------------------------

def _wave_fn(rho, rhoK, cs):
    """velocity change across a left/right wave to star density rho (shock or rarefaction)."""
    if rho > rhoK:
        return cs * (rho - rhoK) / math.sqrt(rho * rhoK)
    return cs * math.log(rho / rhoK)


def exact_isothermal(rhoL, uL, rhoR, uR, cs, xi):
    """density at x/t = xi of the 1D isothermal Riemann problem."""
    lo, hi = 1e-12, 1e6
    for _ in range(300):  # bisection on u*_L(rho) - u*_R(rho) (monotone decreasing)
        mid = math.sqrt(lo * hi)
        g = (uL - _wave_fn(mid, rhoL, cs)) - (uR + _wave_fn(mid, rhoR, cs))
        if g > 0:
            lo = mid
        else:
            hi = mid
    rs = math.sqrt(lo * hi)
    us = uL - _wave_fn(rs, rhoL, cs)
    out = np.empty_like(xi)
    for n, x in enumerate(xi):
        if x < us:  # left of the contact
            if rs > rhoL:
                S = uL - cs * math.sqrt(rs / rhoL)
                out[n] = rhoL if x < S else rs
            else:
                if x < uL - cs:
                    out[n] = rhoL
                elif x > us - cs:
                    out[n] = rs
                else:
                    out[n] = rhoL * math.exp((uL - (x + cs)) / cs)
        else:
            if rs > rhoR:
                S = uR + cs * math.sqrt(rs / rhoR)
                out[n] = rhoR if x > S else rs
            else:
                if x > uR + cs:
                    out[n] = rhoR
                elif x < us + cs:
                    out[n] = rs
                else:
                    out[n] = rhoR * math.exp(((x - cs) - uR) / cs)
    return out


def test_exact_isothermal_riemann_helper():
    # shock tube with a left rarefaction and a right shock: the star state
    # satisfies both wave curves, and the shock obeys the jump conditions
    cs = 1.0
    xi = np.linspace(-3, 3, 2001)
    r = exact_isothermal(2.0, 0.0, 1.0, 0.0, cs, xi)
    assert r[0] == 2.0 and r[-1] == 1.0 and np.all(np.diff(r) <= 1e-12)
    rs = r[np.searchsorted(xi, 0.0)]
    us = -_wave_fn(rs, 2.0, cs)
    assert abs(us - _wave_fn(rs, 1.0, cs)) < 1e-12
    S = cs * math.sqrt(rs)  # right shock speed u_R + cs sqrt(rho*/rho_R) with u_R = 0, rho_R = 1
    # mass and momentum jump conditions across the right shock
    assert abs((rs * (us - S)) - (1.0 * (0.0 - S))) < 1e-12
    assert abs((rs * (us - S) ** 2 + cs * cs * rs) - (1.0 * S * S + cs * cs * 1.0)) < 1e-12


@pytest.mark.parametrize("solver", ["hllc", "rusanov"])
def test_scheme_converges_to_exact_riemann_solution(solver):
    # 1D shock tube along x in the periodic box: rho = 2 on x < 1/2, 1 elsewhere
    # (a second, mirrored problem sits at x = 0); k = 1, SSP-RK2, vNR viscosity.
    # The cell-mean density error against the exact solution falls with N.
    cs, t_end = 1.0, 0.12
    errs = []
    for N in (8, 16):
        k = 1
        b = O.nmodes(k)
        u = np.zeros((N ** 3, 4, b))
        ix = np.arange(N ** 3) % N
        u[:, 0, 0] = np.where(ix < N // 2, 2.0, 1.0)
        cfg = O.make_cfg(N, k, cs=cs, riemann=solver)
        t = 0.0
        while t < t_end:
            rc, t, _, _ = O.run(cfg, u, 1, t=t)
            assert rc == 0
        rho0 = u[:, 0, 0].reshape(N, N, N)
        assert np.abs(rho0 - rho0[:1, :1, :]).max() < 1e-12  # stays one-dimensional
        # cell means of the exact solution by a fine midpoint rule; two
        # non-interacting problems: (2 | 1) at x = 1/2 and (1 | 2) at x = 0 (= 1)
        xf = (np.arange(N * 64) + 0.5) / (N * 64)
        exf = np.where(xf < 0.75, exact_isothermal(2.0, 0.0, 1.0, 0.0, cs, (xf - 0.5) / t),
                       exact_isothermal(1.0, 0.0, 2.0, 0.0, cs, (xf - 1.0) / t))
        exf = np.where(xf < 0.25, exact_isothermal(1.0, 0.0, 2.0, 0.0, cs, xf / t), exf)
        ex = exf.reshape(N, 64).mean(axis=1)
        errs.append(np.abs(rho0[0, 0, :] - ex).mean())
    assert errs[1] < 0.8 * errs[0], errs
    assert errs[1] < 0.06, errs
