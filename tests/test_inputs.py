"""The seeded input recipes (paper_2401_06841_gb300/inputs.py) against what
they promise, by brute force: the turbulent velocity's per-cell coefficients
are the L2 projection of a band-limited Fourier field (its amplitudes
recovered from the cell means alone, then projected cell by cell with a
12-point Gauss rule), the Helmholtz weight zeta selects the transverse or the
longitudinal part, and the rms cell-mean speed is the requested Mach number;
the random parity states keep the density above its stated bound at every
point and the five-variable ones their cell-mean pressure inside its band.
CPU only."""
import numpy as np
import pytest

from paper_2401_06841_gb300 import inputs as I


def legendre_orthonormal(m, x):
    # sqrt(2m+1) P_m(x) by the three-term recurrence
    p0, p1 = np.ones_like(x), x
    if m == 0:
        return p0
    for j in range(2, m + 1):
        p0, p1 = p1, ((2 * j - 1) * x * p1 - (j - 1) * p0) / j
    return np.sqrt(2 * m + 1) * p1


def amplitudes_from_means(means, N):
    # cell means of sum_k a_k exp(2 pi i k.x) are a_k prod_d sinc(pi k_d h)
    # sampled at the centres x_c = (i + 1/2) h: invert that on the lattice
    F = np.fft.fftn(means.reshape(N, N, N))
    kk = np.fft.fftfreq(N, d=1.0 / N)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    h = 1.0 / N
    S = np.sinc(KX * h) * np.sinc(KY * h) * np.sinc(KZ * h)  # numpy sinc(x) = sin(pi x)/(pi x)
    return F * np.exp(-1j * np.pi * (KX + KY + KZ) / N) / (N ** 3 * S), (KX, KY, KZ)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_turbulent_velocity_is_the_projection_of_its_fourier_field(k):
    N = 8  # band 2 <= |kappa| <= N/4 = 2: the six axis wave vectors
    u = I.turbulent_velocity(N, k, seed=4, mach=1.5, zeta=0.5)
    ijl = I.mode_degrees(k)
    h = 1.0 / N
    xg, wg = np.polynomial.legendre.leggauss(12)
    rng = np.random.default_rng(0)
    cells = rng.choice(N ** 3, 12, replace=False)
    for comp in range(3):
        a, (KX, KY, KZ) = amplitudes_from_means(u[:, comp, 0], N)
        keep = np.abs(a) > 1e-12 * np.abs(a).max()
        kv = np.stack([KX[keep], KY[keep], KZ[keep]], axis=1)
        norms = np.sqrt((kv ** 2).sum(axis=1))
        assert np.all((norms >= 2 - 1e-12) & (norms <= 2 + 1e-12))  # the band
        av = a[keep]
        for c in cells:
            iz, iy, ix = c // (N * N), (c // N) % N, c % N
            # points of the 12^3 Gauss rule in cell c
            X = (ix + 0.5 + 0.5 * xg) * h
            Y = (iy + 0.5 + 0.5 * xg) * h
            Z = (iz + 0.5 + 0.5 * xg) * h
            ex = np.exp(2j * np.pi * np.outer(kv[:, 0], X))  # [modes][12]
            ey = np.exp(2j * np.pi * np.outer(kv[:, 1], Y))
            ez = np.exp(2j * np.pi * np.outer(kv[:, 2], Z))
            # field at the points, indexed [z][y][x]
            f = np.einsum("m,mz,my,mx->zyx", av, ez, ey, ex).real
            w = wg / 2.0
            for l, (i, j, lz) in enumerate(ijl):
                px = legendre_orthonormal(i, xg)
                py = legendre_orthonormal(j, xg)
                pz = legendre_orthonormal(lz, xg)
                coef = np.einsum("zyx,z,y,x->", f, w * pz, w * py, w * px)
                assert u[c, comp, l] == pytest.approx(coef, abs=1e-12 * np.abs(u[:, comp]).max()), (comp, c, l)


@pytest.mark.parametrize("zeta", [0.0, 1.0])
def test_helmholtz_weight_selects_the_part(zeta):
    # zeta = 1: transverse (k . a_k = 0); zeta = 0: longitudinal (k x a_k = 0),
    # checked on the amplitudes recovered from the cell means
    N, k = 16, 1
    u = I.turbulent_velocity(N, k, seed=11, mach=1.0, zeta=zeta)
    a = []
    for comp in range(3):
        ac, (KX, KY, KZ) = amplitudes_from_means(u[:, comp, 0], N)
        a.append(ac)
    a = np.stack(a)
    kv = np.stack([KX, KY, KZ])
    scale = np.abs(a).max() * np.abs(kv).max()
    if zeta == 1.0:
        assert np.abs((kv * a).sum(axis=0)).max() < 1e-10 * scale
    else:
        cross = np.cross(kv, a, axis=0)
        assert np.abs(cross).max() < 1e-10 * scale
    assert np.abs(a).max() > 0


def test_rms_cell_mean_speed_is_the_mach_number():
    for mach, cs in ((0.5, 1.0), (3.0, 2.0)):
        v = I.turbulent_velocity(8, 2, seed=3, mach=mach, cs=cs)
        assert np.sqrt((v[:, :, 0] ** 2).sum(axis=1).mean()) == pytest.approx(mach * cs, rel=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_random_state_density_stays_above_its_bound(k):
    # sum_l |rho_l| sup|phi_l| = wiggle * rho_0 for the higher modes, so at
    # any point of the cell rho >= (1 - wiggle) rho_0: sampled at random points
    N, wiggle = 4, 0.6
    u = I.random_state(N, k, seed=21 + k, rho_wiggle=wiggle)
    rng = np.random.default_rng(k)
    xi = rng.uniform(-1, 1, (3, 4000))
    ijl = I.mode_degrees(k)
    phi = np.stack([legendre_orthonormal(i, xi[0]) * legendre_orthonormal(j, xi[1]) * legendre_orthonormal(l, xi[2])
                    for (i, j, l) in ijl])  # [b][points]
    rho = u[:, 0, :] @ phi  # [cells][points]
    r0 = u[:, 0, 0][:, None]
    assert (rho >= (1 - wiggle) * r0 - 1e-12).all()
    assert (rho <= (1 + wiggle) * r0 + 1e-12).all()
    # and the bound is not loose: the sampled dip below rho_0 reaches at
    # least 40% of it (random points rarely hit the corner where it is attained)
    assert ((r0 - rho) / r0).max() > 0.4 * wiggle


def test_random_energy_state_cell_mean_pressure():
    # cell-mean pressure (gamma-1)(e_0 - |m_0|^2 / (2 rho_0)) inside p_mean [1 -+ spread/2]
    g, pm, sp = 1.4, 5.0, 0.5
    u = I.random_energy_state(6, 2, seed=8, p_mean=pm, p_spread=sp, gamma=g, v_rms=0.4)
    p = (g - 1) * (u[:, 4, 0] - 0.5 * (u[:, 1:4, 0] ** 2).sum(axis=1) / u[:, 0, 0])
    assert p.min() >= pm * (1 - sp / 2) - 1e-12 and p.max() <= pm * (1 + sp / 2) + 1e-12
    assert p.max() - p.min() > 0.5 * pm * sp  # spread over the band
    ref = I.random_state(6, 2, seed=8, v_rms=0.4)
    assert np.array_equal(u[:, :4], ref)  # rho and m as the isothermal recipe draws them


def test_device_turbulent_state_equals_the_numpy_recipe():
    # the torch build of the turbulent start state (used for the 256^3 benchmark)
    # draws the same numbers and follows the same recipe as turbulent_state
    torch = pytest.importorskip("torch")
    for N, k, zeta in [(8, 3, 0.3), (12, 2, 1.0)]:
        a = I.turbulent_state(N, k, seed=5, mach=2.0, zeta=zeta)
        b = I.turbulent_state_device(N, k, seed=5, mach=2.0, zeta=zeta, device="cpu", dtype=torch.float64).numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
