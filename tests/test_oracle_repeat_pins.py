"""Pins of the oracle's positivity by repetition of the step (Sec. 3.1, last
paragraph, read as the troubled-cell procedure the same section gives for the
finite-volume scheme).

The flagged step is checked against the SSP-RK stages rebuilt here from the
oracle's right-hand side and limiter, with the densities and wave speeds at the
Gauss points evaluated independently (numpy's Legendre series); the repeated
step against the plain step from the flattened input it reports; the halving of
dt on a flat cell with negative density and the failure rule (a mean that is not
positive) against hand-built states; and the whole procedure
against the driven start from rest that the plain rescaling does not survive.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I

RK3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def pnorm(m, x):
    c = np.zeros(m + 1)
    c[m] = 1.0
    return math.sqrt(2 * m + 1) * npleg.legval(x, c)


def point_tables(k):
    """phi at the (k+1)^3 volume Gauss points and at the 6 (k+1)^2 face points."""
    x, _ = np.polynomial.legendre.leggauss(k + 1)
    vol = [(a, b, c) for c in x for b in x for a in x]
    face = []
    for d in range(3):
        for s in (-1.0, 1.0):
            for p in x:
                for q in x:
                    r = [p, q]
                    r.insert(d, s)
                    face.append(tuple(r))
    ijl = I.mode_degrees(k)

    def tab(pts):
        return np.array([[pnorm(i, p[0]) * pnorm(j, p[1]) * pnorm(m, p[2]) for (i, j, m) in ijl] for p in pts])

    return tab(vol), tab(face)


def driven_start(N, k, nsteps, seed=11):
    """The plain scheme from rest (rho = 1, v = 0) under Mach-3 OU driving."""
    cfg = O.make_cfg(N, k)
    u = np.zeros((N ** 3, 4, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    fo = O.Forcing(mach=3.0, zeta=0.5, seed=seed)
    rc, t, _, ah = O.run(cfg, u, nsteps, forcing=fo)
    assert rc == 0
    return cfg, u, ah, fo, t


def brute_flags(cfg, u, ah, dt, vlim):
    """The SSP-RK3 stages from the oracle's rhs and limiter; a cell is marked
    MARK_NEGATIVE when a stage output has rho < 0 at a volume or face point
    (before the limiter) and MARK_FAST when, after it, a volume point has
    sum_d(|v_d| + cs) > vlim."""
    Pv, Pf = point_tables(cfg.k)
    P = np.vstack([Pv, Pf])
    un = u.copy()
    us = u.copy()
    flag = np.zeros(u.shape[0], dtype=np.uint8)
    smax = np.zeros(u.shape[0])
    for a, b in RK3:
        L = O.rhs(cfg, us, ah, dt)
        us = a * un + b * (us + dt * L)
        flag[(us[:, 0] @ P.T).min(1) < 0.0] |= O.MARK_NEGATIVE
        O.limit(cfg, us)
        rv = us[:, 0] @ Pv.T
        sp = sum(np.abs(us[:, 1 + d] @ Pv.T / rv) + cfg.cs for d in range(3)).max(1)
        smax = np.maximum(smax, sp)
        flag[sp > vlim] |= O.MARK_FAST
    return us, flag, smax


def test_flagged_step_marks_the_cells_its_stages_trouble():
    cfg, u, ah, _, _ = driven_start(8, 2, 40)
    dt = O.dt(cfg, u)
    # positivity marks alone
    ref, fref, smax = brute_flags(cfg, u, ah, dt, 1e300)
    w = u.copy()
    st, flag = O.step_flags(cfg, w, ah, dt, 1e300)
    assert (fref == O.MARK_NEGATIVE).any() and (st & O.ST_LIMITED)
    np.testing.assert_array_equal(flag, fref)
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-12)
    # wave-speed marks: a bound between two cells' stage maxima marks the faster half
    s = np.sort(smax)
    vlim = 0.5 * (s[len(s) // 2] + s[len(s) // 2 + 1])
    _, fref2, _ = brute_flags(cfg, u, ah, dt, vlim)
    _, flag2 = O.step_flags(cfg, u.copy(), ah, dt, vlim)
    assert ((fref2 & O.MARK_FAST) != 0).sum() == len(s) - len(s) // 2 - 1
    np.testing.assert_array_equal(flag2, fref2)


def test_repetition_is_the_plain_step_when_no_cell_is_troubled():
    N, k = 4, 2
    cfg = O.make_cfg(N, k)
    cfgr = O.make_cfg(N, k, positivity="repeat")
    u = I.sound_wave(N, k, eps=1e-3, kvec=(1, 1, 0))
    assert np.isfinite(u).all()
    ref = u.copy()
    O.step(cfg, ref, None, O.dt(cfg, u))
    w = u.copy()
    st, dtu, att, lev = O.step_repeat(cfgr, w, None)
    assert st >= 0 and not (st & O.ST_REPEATED) and att == 1 and not lev.any()
    assert dtu == O.dt(cfg, u)
    np.testing.assert_array_equal(w, ref)


@pytest.mark.parametrize("k,nsteps", [(2, 40), (1, 60)])  # SSP-RK3 and SSP-RK2
def test_repetition_is_the_plain_step_from_the_flattened_input(k, nsteps):
    cfg, u, ah, _, _ = driven_start(8, k, nsteps)
    cfgr = O.make_cfg(8, k, positivity="repeat")
    w = u.copy()
    st, dtu, att, lev = O.step_repeat(cfgr, w, ah)
    assert st >= 0 and (st & O.ST_REPEATED) and att >= 2 and lev.any()
    # u^n with every troubled cell's modes l > 0 scaled 1/2, 1/4, then 0
    f = np.array([1.0, 0.5, 0.25, 0.0])[lev]
    uf = u.copy()
    uf[:, :, 1:] *= f[:, None, None]
    h = math.log2(O.dt(cfg, uf) / dtu)
    assert h == round(h) and 0 <= h <= 6
    ref = uf.copy()
    st_ref = O.step(cfgr, ref, ah, dtu)
    np.testing.assert_array_equal(w, ref)
    assert not (st_ref & O.ST_FAIL)
    # the accepted step troubles no cell but flat ones for their speed; no point is
    # negative, and the cells whose mean is above the floor have every point at it
    # or above (the rescaling)
    _, flag = O.step_flags(cfg, uf.copy(), ah, dtu, O.REPEAT_SPEED * O.speed_bound(cfg, uf))
    flat = ~np.any(uf[:, :, 1:] != 0.0, axis=(1, 2))
    assert not (flag & O.MARK_NEGATIVE).any() and not (flag.astype(bool) & ~flat).any()
    Pv, Pf = point_tables(k)
    pts = (w[:, 0] @ np.vstack([Pv, Pf]).T).min(1)
    assert pts.min() >= 0.0
    assert (pts[w[:, 0, 0] > cfg.rho_floor] >= cfg.rho_floor * (1 - 1e-12)).all()
    # scaling higher modes keeps the cell means: the mass is that of u^n
    assert abs(w[:, 0, 0].sum() - u[:, 0, 0].sum()) < 1e-12 * u[:, 0, 0].sum()


def _diverging_pair(N, k, rho0, V=3.0):
    """Flat cells of density rho0 at rest but cell c, moving along +x, and its
    left neighbour, moving along -x: c drains through its +x face."""
    c = (2 * N + 2) * N + 2                     # cell (2, 2, 2)
    u = I.uniform_state(N, k, rho=rho0)
    u[c - 1, 1, 0] = -V * rho0
    u[c, 1, 0] = V * rho0
    return u, c


def test_a_flat_cell_with_negative_density_halves_dt():
    # with a prescribed dt of four CFL steps the two flat moving cells end with
    # negative density; flat cells cannot be scaled, so dt is halved, and the
    # step at half of it troubles no cell
    N, k = 6, 1
    cfgr = O.make_cfg(N, k, positivity="repeat")
    u, c = _diverging_pair(N, k, 1.0)
    dt4 = 4.0 * O.dt(cfgr, u)
    _, flag = O.step_flags(cfgr, u.copy(), None, dt4, 1e300)
    np.testing.assert_array_equal(np.nonzero(flag)[0], [c - 1, c])
    assert (flag[[c - 1, c]] == O.MARK_NEGATIVE).all()
    w = u.copy()
    st, dtu, att, lev = O.step_repeat(cfgr, w, None, fixed_dt=dt4)
    assert st >= 0 and (st & O.ST_REPEATED) and att == 2 and not lev.any()
    assert dtu == 0.5 * dt4
    ref = u.copy()
    O.step(cfgr, ref, None, dtu)
    np.testing.assert_array_equal(w, ref)


def test_only_a_non_positive_mean_fails_the_repetition():
    # the step is linear in rho0 (fluxes and Pi are; dt is not affected), so the
    # fraction f that c loses in a CFL step, measured at rho0 = 1, fixes a rho0
    # whose step ends with c's mean in (0, floor): a failure for the rescaling
    # (dt halved, at most 3 times), a state that stands for the repetition
    N, k = 6, 1
    cfg = O.make_cfg(N, k)
    cfgr = O.make_cfg(N, k, positivity="repeat")
    u1, c = _diverging_pair(N, k, 1.0)
    dt0 = O.dt(cfg, u1)
    a = u1.copy()
    O.step(cfg, a, None, dt0)
    f = 1.0 - a[c, 0, 0]
    assert 0.0 < f < 0.5
    u, _ = _diverging_pair(N, k, cfg.rho_floor / (1.0 - 0.5 * f))
    assert O.step(cfg, u.copy(), None, dt0) & O.ST_FAIL
    w = u.copy()
    st, dtu, att, lev = O.step_repeat(cfgr, w, None)
    assert st >= 0 and not (st & O.ST_FAIL) and att == 1 and dtu == dt0
    assert 0.0 < w[c, 0, 0] < cfg.rho_floor
    ref = u.copy()
    O.step(cfgr, ref, None, dt0)
    np.testing.assert_array_equal(w, ref)


@pytest.mark.timeout(300)
def test_repetition_survives_the_driven_start_that_the_rescaling_does_not():
    # the plain rescaling: a velocity spike at a limited point after t ~ 0.09
    cfg, u, ah, fo, t = driven_start(8, 2, 40)
    rc, t1, _, _ = O.run(cfg, u, 10, forcing=fo, t=t, ahat=ah)
    assert rc != 0 or not np.isfinite(u).all() or O.speed_bound(cfg, u) > 1e3
    # the repetition from the same start reaches t = 0.15 with bounded speeds
    N, k = 8, 2
    cfgr = O.make_cfg(N, k, positivity="repeat")
    u = np.zeros((N ** 3, 4, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    fo = O.Forcing(mach=3.0, zeta=0.5, seed=11)
    t, ah, steps = 0.0, None, 0
    while t < 0.15 and steps < 2000:
        rc, t, _, ah = O.run(cfgr, u, 10, forcing=fo, t=t, ahat=ah)
        steps += 10
        assert rc == 0 and np.isfinite(u).all()
    assert t >= 0.15
    assert O.speed_bound(cfgr, u) < 60.0
    assert abs(u[:, 0, 0].mean() - 1.0) < 1e-12
