"""Pins of the oracle's turbulence statistics (Sec. 4.1 structure function and
power spectrum, Sec. 4.3 sampling, density PDF) against closed forms: a
density with a known distribution over each cell, and a single Fourier mode
whose structure function and spectrum are known exactly."""
import math

import numpy as np
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2401_06841_gb300 import inputs as I


def test_density_pdf_of_a_linear_profile():
    # rho = 1 + a xi_x in every cell (mean 1): the Gauss points of a cell carry
    # rho_a = 1 + a x_a with volume fraction w_a / 2 each
    N, k, a = 3, 2, 0.6
    b = O.nmodes(k)
    ml = [tuple(r) for r in O.mode_list(k)]
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, 0] = 1.0
    u[:, 0, ml.index((1, 0, 0))] = a / math.sqrt(3.0)
    lo, hi, nb = -0.5, 0.5, 200
    h = O.density_pdf(O.make_cfg(N, k), u, lo, hi, nb)
    x, w = npleg.leggauss(k + 1)
    ref = np.zeros(nb)
    for xa, wa in zip(x, w):
        ref[int(math.floor((math.log10(1 + a * xa) - lo) / ((hi - lo) / nb)))] += wa / 2
    assert np.allclose(h, ref, atol=1e-14)
    # a uniform state puts the whole volume in the bin of log10(1) = 0
    u[:, 0, ml.index((1, 0, 0))] = 0.0
    h0 = O.density_pdf(O.make_cfg(N, k), u, lo, hi, nb)
    assert abs(h0[nb // 2] - 1.0) < 1e-14 and abs(h0.sum() - 1.0) < 1e-14


def single_mode(N, k, A):
    """rho = 1, v_y = A sin(2 pi x) (exact L2 coefficients)."""
    b = O.nmodes(k)
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, 0] = 1.0
    u[:, 2, :] = A * I.fourier_coeffs(N, k, (1, 0, 0)).imag
    return u


def test_structure_function_of_a_single_mode():
    # |v(x) - v(x + l n)|^2 averaged over x and over directions n on the sphere:
    # A^2 (1 - <cos(2 pi l n_x)>) = A^2 (1 - sin(2 pi l) / (2 pi l))
    N, k, A = 8, 3, 0.7
    u = single_mode(N, k, A)
    nb, npairs = 12, 4000
    l, v = O.structure_function(O.make_cfg(N, k), u, nb, npairs, seed=5)
    lmin = 1.0 / ((k + 1) * N)
    assert np.allclose(l, lmin * (0.5 / lmin) ** ((np.arange(nb) + 0.5) / nb), rtol=1e-14)
    ref = np.sqrt(0.5 * A * A * (1 - np.sin(2 * np.pi * l) / (2 * np.pi * l)))
    # Monte Carlo with 4000 pairs: a few per cent
    assert np.all(np.abs(v / ref - 1) < 0.06), v / ref
    # large separations approach the rms velocity (Sec. 4.1): v(l)^2 -> <v^2> = A^2/2
    assert abs(v[-1] ** 2 / (A * A / 2) - 1) < 0.25


def test_power_spectrum_of_a_single_mode_and_parseval():
    N, k, A = 6, 2, 0.5
    u = single_mode(N, k, A)
    cfg = O.make_cfg(N, k)
    kmean, power, count = O.power_spectrum(cfg, u, 40)
    # all power sits at |kappa| = 1 (the first bin holds the 6 unit vectors), A^2/2
    assert count[0] == 6 and kmean[0] == 1.0
    assert abs(power[0] / (A * A / 2) - 1) < 1e-3
    assert power[1:].sum() < 1e-4 * power[0]  # the P_2 representation of the sine leaks ~h^6
    # Parseval: the bins add up to the variance of the sampled field
    v = O.sample_velocity(cfg, u)
    var = sum((v[d] ** 2).mean() - v[d].mean() ** 2 for d in range(3))
    assert abs(power.sum() - var) < 1e-12 * var
    Ng = (k + 1) * N
    assert count.sum() == Ng ** 3 - 1
    # the sampled field is the DG velocity at cell-interior grid points
    xg = (np.arange(Ng) + 0.5) / Ng
    # (P_2 on h = 1/6: pointwise error ~1e-3; a grid shifted by half a spacing would be off by ~0.09)
    assert np.abs(v[1][0, 0, :] - A * np.sin(2 * np.pi * xg)).max() < 3e-3
