"""Pins of the oracle's diagnostics (Sec. 4.1, Sec. 4.2) and of its driving
schedule (Sec. 4.2) against closed forms.

Diagnostics: every state below is written out coefficient by coefficient in
each cell's reference coordinate xi, so that each reported quantity has a value
worked out by hand from cell averages of powers of xi (<xi> = <xi^3> = 0,
<xi^2> = 1/3).  The states are chosen so that the plausible mistakes give other
numbers: volume- and mass-weighted Mach numbers differ, the mass-weighted mean
acceleration differs from the volume mean and from zero, part of the volume is
compressed above the sensor threshold, part below it and part expanded.

Driving schedule: the OU variables after every step of a run are compared,
bit for bit, with a separate OU process of the same seed advanced by hand the
number of times the schedule prescribes (one update at the start of every step
for each multiple of t_c/100 that the time has reached, none at t = 0).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def modes(k):
    return [tuple(int(v) for v in r) for r in O.mode_list(k)]


def cls_of(N):
    """cell index -> (ix, iy, iz)"""
    c = np.arange(N ** 3)
    return c % N, (c // N) % N, c // (N * N)


# polynomials of the cell coordinate xi_x in the orthonormal basis:
#   1 = phi_000,  xi = phi_100 / sqrt3,  xi^2 = 1/3 + 2 phi_200 / (3 sqrt5)
def set_poly(u, cells, var, k, c0=0.0, c1=0.0, c2=0.0):
    """u[cells, var] = c0 + c1 xi_x + c2 xi_x^2"""
    ml = modes(k)
    u[cells, var, ml.index((0, 0, 0))] = c0 + c2 / 3.0
    u[cells, var, ml.index((1, 0, 0))] = c1 / math.sqrt(3.0)
    if c2 != 0.0:
        u[cells, var, ml.index((2, 0, 0))] = c2 * 2.0 / (3.0 * math.sqrt(5.0))


def test_mach_numbers_volume_and_mass_weighted():
    # half of the cells rho = 1, v_x = 0.4; the other half rho = 3, v_x = -0.2
    # (constant in each cell).  M^2 = <v^2>/cs^2 (volume mean), M_rho^2 =
    # <rho v^2>/<rho> / cs^2 (mass weighted): 0.1/cs^2 and 0.07/cs^2.
    N, k, cs = 2, 1, 0.5
    b = O.nmodes(k)
    u = np.zeros((N ** 3, 4, b))
    ix, _, _ = cls_of(N)
    light, heavy = ix == 0, ix == 1
    u[light, 0, 0], u[light, 1, 0] = 1.0, 0.4
    u[heavy, 0, 0], u[heavy, 1, 0] = 3.0, 3.0 * -0.2
    d = O.diagnostics(O.make_cfg(N, k, cs=cs), u)
    assert d["mass"] == pytest.approx(2.0, rel=1e-14)
    assert d["mom_x"] == pytest.approx((0.4 - 0.6) / 2, rel=1e-13)
    assert d["mom_y"] == 0.0 and d["mom_z"] == 0.0
    assert d["ekin"] == pytest.approx(0.5 * (1 * 0.16 + 3 * 0.04) / 2, rel=1e-13)
    assert d["mach"] == pytest.approx(math.sqrt((0.16 + 0.04) / 2) / cs, rel=1e-13)
    assert d["mach_rho"] == pytest.approx(math.sqrt((0.16 + 3 * 0.04) / 4) / cs, rel=1e-13)
    assert d["rho_min"] == pytest.approx(1.0) and d["rho_max"] == pytest.approx(3.0)
    assert d["max_speed"] == pytest.approx(0.4 + 3 * cs, rel=1e-14)
    assert d["av_frac"] == 0.0 and d["av_work"] == 0.0


def test_injected_power_uses_the_mass_weighted_mean_acceleration():
    # every cell: rho = 2 + al xi, v_x = V xi (m_x = 2 V xi + al V xi^2), a_x = be xi + ga.
    # abar_x = <rho a_x>/<rho> = ga + al be/6 (mass weighted; the volume mean is ga, the
    # unnormalised <rho a_x> is 2 ga + al be/3), and int m.(a - abar) = V be (2/3 - al^2/18).
    # Without abar it would be V (2 be + ga al)/3, with the volume mean 2 V be/3.
    N, k = 2, 2
    al, V, be, ga = 0.5, 0.3, 0.2, 0.7
    b = O.nmodes(k)
    cells = np.arange(N ** 3)
    u = np.zeros((N ** 3, 4, b))
    set_poly(u, cells, 0, k, 2.0, al)
    set_poly(u, cells, 1, k, 0.0, 2 * V, al * V)
    ah = np.zeros((N ** 3, 3, b))
    set_poly(ah, cells, 0, k, ga, be)
    cfg = O.make_cfg(N, k)
    assert O.forcing_mean(cfg, u, ah) == pytest.approx([ga + al * be / 6, 0.0, 0.0], rel=1e-14, abs=1e-16)
    d = O.diagnostics(cfg, u, ah)
    assert d["inj_power"] == pytest.approx(V * be * (2 / 3 - al * al / 18), rel=1e-13)
    # rho v^2 = V^2 xi^2 (2 + al xi): E_kin = V^2/3, <v^2> = V^2/3; the gas expands (no AV)
    assert d["mass"] == pytest.approx(2.0, rel=1e-14)
    assert d["ekin"] == pytest.approx(V * V / 3, rel=1e-13)
    assert d["mach"] == pytest.approx(V / math.sqrt(3), rel=1e-13)
    assert d["av_frac"] == 0.0 and d["av_work"] == 0.0


def test_viscous_fraction_and_work_on_compressed_cells():
    # rho = 1 and v_x = -c (h/2) xi (div v = -c) with three values of c by cell:
    # strong compression c = 4 (half of the volume), weak compression c = 0.2 (a quarter)
    # and expansion c = -4 (a quarter).  vNR (Sec. 3.1, dt = 0: no cap):
    # Pi = al rho (h/p)^2 c^2 + be rho cs (h/p) c, counted in av_frac where Pi > 0.01 cs^2 rho
    # (only the strong class: Pi_weak = 0.0089); av_work = int Pi div v.
    N, k, cs = 2, 2, 1.0
    h, hp = 1.0 / N, 1.0 / N / (k + 1)
    b = O.nmodes(k)
    ix, iy, _ = cls_of(N)
    cls = {4.0: ix == 0, 0.2: (ix == 1) & (iy == 0), -4.0: (ix == 1) & (iy == 1)}
    u = np.zeros((N ** 3, 4, b))
    for c, sel in cls.items():
        set_poly(u, sel, 0, k, 1.0)
        set_poly(u, sel, 1, k, 0.0, -c * h / 2)
    d = O.diagnostics(O.make_cfg(N, k, cs=cs), u)

    def vnr(c):
        return 2.0 * hp * hp * c * c + 0.2 * cs * hp * c if c > 0 else 0.0

    assert vnr(0.2) < 0.01 * cs * cs < vnr(4.0)
    assert d["av_frac"] == pytest.approx(0.5, rel=1e-14)
    frac = {4.0: 0.5, 0.2: 0.25, -4.0: 0.25}
    assert d["av_work"] == pytest.approx(sum(f * vnr(c) * -c for c, f in frac.items()), rel=1e-13)
    # E_kin = (1/2) <v^2> = (1/2) c^2 h^2 / 12 per class
    assert d["ekin"] == pytest.approx(sum(f * c * c * h * h / 24 for c, f in frac.items()), rel=1e-13)
    # the cap with a step dt: Pi <= rho (h/p)^2 |div v| / (2 dt)
    dt = 0.1
    dc = O.diagnostics(O.make_cfg(N, k, cs=cs), u, None, dt)
    pmax = lambda c: min(vnr(c), 0.5 * hp * hp * c / dt)  # noqa: E731
    assert pmax(4.0) < vnr(4.0) and pmax(0.2) == vnr(0.2)
    assert dc["av_work"] == pytest.approx(0.5 * pmax(4.0) * -4.0 + 0.25 * pmax(0.2) * -0.2, rel=1e-13)


def _run_stepwise(cfg, u, fo, nsteps):
    """advance one step at a time; returns the time at the start of each step,
    and the OU variables and projected forcing after it"""
    t, ah = 0.0, None
    ts, xs, ahs, us = [], [], [], [u.copy()]
    for _ in range(nsteps):
        ts.append(t)
        rc, t, _, ah = O.run(cfg, u, 1, forcing=fo, t=t, ahat=ah)
        assert rc == 0
        xs.append(fo.x())
        ahs.append(ah.copy())
        us.append(u.copy())
    return ts, t, xs, ahs, us


def test_ou_update_schedule_counts_the_advances():
    # t_c = 1/(2 cs M) = 1 at M = 0.5, so dt_drive = 0.01 against dt ~ 0.025 (N = 2, k = 1):
    # two or three OU updates per step.  At the start of a step with time t the process
    # has been advanced once for every j >= 1 with j dt_drive <= t.
    N, k, mach, seed = 2, 1, 0.5, 5
    cfg = O.make_cfg(N, k)
    fo = O.Forcing(mach=mach, zeta=0.5, seed=seed)
    dtd = fo.ou.dt_drive
    assert dtd == pytest.approx(0.01, rel=1e-15)
    u = np.zeros((N ** 3, 4, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    ts, t_end, xs, ahs, _ = _run_stepwise(cfg, u, fo, 8)
    ref = O.Forcing(mach=mach, zeta=0.5, seed=seed)
    done = 0
    counts = []
    for t, x, ah in zip(ts, xs, ahs):
        # no step starts within round-off of an update time
        assert abs(t / dtd - round(t / dtd)) > 1e-9 or t == 0.0
        want = int(math.floor(t / dtd + 1e-12))
        while done < want:
            ref.advance()
            done += 1
        counts.append(want)
        assert np.array_equal(x, ref.x())
        assert np.array_equal(ah, O.forcing_project(cfg, ref.kvec(), ref.amplitudes()))
    # the first step drives with the initial (stationary) draw; later steps see 2-3 updates
    assert counts[0] == 0 and counts[1] == 2
    assert all(2 <= b - a <= 3 for a, b in zip(counts, counts[1:]))
    assert counts[-1] == int(math.floor(ts[-1] / dtd))


def test_ou_driving_stops_after_t_off():
    # with t_off the process is advanced only while t <= t_off, and after it the
    # steps are undriven: the OU variables stay at their last values
    N, k, mach, seed = 2, 1, 0.5, 6
    cfg = O.make_cfg(N, k)
    t_off = 0.06
    fo = O.Forcing(mach=mach, zeta=0.5, seed=seed, t_off=t_off)
    u = np.zeros((N ** 3, 4, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    ts, _, xs, _, us = _run_stepwise(cfg, u, fo, 6)
    ref = O.Forcing(mach=mach, zeta=0.5, seed=seed)
    last_on = max(i for i, t in enumerate(ts) if t <= t_off)
    assert 0 < last_on < len(ts) - 1
    for _ in range(int(math.floor(ts[last_on] / fo.ou.dt_drive + 1e-12))):
        ref.advance()
    for i in range(last_on, len(ts)):
        assert np.array_equal(xs[i], ref.x())
    assert fo.ou.on == 0
    # a step that starts after t_off is an undriven step of the same state, bit for bit,
    # and the last step before it is not
    for i in (last_on, last_on + 1):
        u2 = us[i].copy()
        rc, _, _, _ = O.run(cfg, u2, 1, t=ts[i])
        assert rc == 0
        assert np.array_equal(u2, us[i + 1]) == (i > last_on)
