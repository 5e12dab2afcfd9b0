"""Seeded synthetic inputs for the DG solver, shared by the tests, the smoke check
and the benchmark.

This module holds no step of the method: no quadrature rule, no flux, no
projection by quadrature.  It only produces modal coefficient arrays in the
library's layout ``u[cell][var][mode]`` (cell = (iz*N + iy)*N + ix, var =
rho, m_x, m_y, m_z, modes of the complete degree-k set of normalised Legendre
products ordered by total degree, then i descending, then j descending), by
two routes:

* ``random_state``: independent random coefficients per cell (discontinuous
  across cells), with a density kept positive by construction;
* ``fourier_coeffs``: the EXACT L2 coefficients of a plane wave
  exp(2 pi i kappa . x) on every cell, from the closed form
  (1/2) int_{-1}^{1} P_m(t) exp(i a t) dt = i^m j_m(a)  (spherical Bessel j_m),
  so band-limited fields (sound waves, synthetic turbulence) can be set up
  without any quadrature.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn


def nmodes(k: int) -> int:
    return (k + 1) * (k + 2) * (k + 3) // 6


def mode_degrees(k: int) -> np.ndarray:
    """(i, j, l) Legendre degrees of each mode in the library's order."""
    out = []
    for d in range(k + 1):
        for i in range(d, -1, -1):
            for j in range(d - i, -1, -1):
                out.append((i, j, d - i - j))
    return np.array(out, dtype=np.int64)


def basis_sup(k: int) -> np.ndarray:
    """max over the reference cube of |phi_l| = prod sqrt(2m+1) (|P_m| <= 1)."""
    ijl = mode_degrees(k)
    return np.sqrt((2 * ijl + 1).prod(axis=1).astype(np.float64))


def random_state(N: int, k: int, seed: int, rho_mean: float = 1.0, rho_spread: float = 0.5,
                 rho_wiggle: float = 0.6, v_rms: float = 0.5, decay: float = 0.6) -> np.ndarray:
    """Random per-cell modal coefficients.

    Cell means of rho are uniform in rho_mean*[1-rho_spread/2, 1+rho_spread/2];
    the higher rho modes are Gaussian, rescaled per cell so that
    sum_l |rho_l| max|phi_l| = rho_wiggle * rho_0 (< rho_0), which keeps rho > 0
    at every point of the cell.  Momentum modes are rho_0 times Gaussian
    velocities of rms v_rms, damped by decay**degree.
    """
    rng = np.random.default_rng(seed)
    b = nmodes(k)
    nc = N ** 3
    deg = mode_degrees(k).sum(axis=1)
    u = np.zeros((nc, 4, b))
    r0 = rho_mean * (1.0 + rho_spread * (rng.random(nc) - 0.5))
    u[:, 0, 0] = r0
    if b > 1:
        hi = rng.standard_normal((nc, b - 1)) * decay ** deg[1:]
        s = (np.abs(hi) * basis_sup(k)[1:]).sum(axis=1)
        u[:, 0, 1:] = hi * (rho_wiggle * r0 / np.maximum(s, 1e-300))[:, None]
    for i in range(3):
        u[:, 1 + i, :] = rng.standard_normal((nc, b)) * v_rms * decay ** deg * r0[:, None]
    return u


def _axis_factors(N: int, k: int, kap: int) -> np.ndarray:
    """[N][k+1] complex: exp(2 pi i kap x_c) sqrt(2m+1) i^m j_m(pi kap h) for each cell centre."""
    h = 1.0 / N
    xc = (np.arange(N) + 0.5) * h
    a = np.pi * kap * h
    m = np.arange(k + 1)
    g = np.sqrt(2 * m + 1) * (1j ** m) * spherical_jn(m, a)
    return np.exp(2j * np.pi * kap * xc)[:, None] * g[None, :]


def random_energy_state(N: int, k: int, seed: int, p_mean: float = 1.5, p_spread: float = 0.5,
                        wiggle: float = 0.05, gamma: float = 1.4, **kw) -> np.ndarray:
    """Random coefficients [N^3][5][b] for a five-variable state (rho, m, e):
    rho and m from ``random_state`` (same seed and keywords); the cell mean of
    e gives a mean pressure p uniform in p_mean*[1-p_spread/2, 1+p_spread/2]
    with the cell-mean kinetic energy density |m_0|^2/(2 rho_0); the higher
    modes of e are Gaussian, wiggle * e_0 times decay**degree."""
    u4 = random_state(N, k, seed, **kw)
    rng = np.random.default_rng(seed + 7919)
    b = nmodes(k)
    nc = N ** 3
    deg = mode_degrees(k).sum(axis=1)
    u = np.zeros((nc, 5, b))
    u[:, :4] = u4
    p0 = p_mean * (1.0 + p_spread * (rng.random(nc) - 0.5))
    e0 = p0 / (gamma - 1.0) + 0.5 * (u4[:, 1:, 0] ** 2).sum(axis=1) / u4[:, 0, 0]
    u[:, 4, 0] = e0
    if b > 1:
        u[:, 4, 1:] = rng.standard_normal((nc, b - 1)) * wiggle * kw.get("decay", 0.6) ** deg[1:] * e0[:, None]
    return u


def adiabatic_turbulent_state(N: int, k: int, seed: int, mach: float, gamma: float = 1.4, p0: float = 1.0,
                              zeta: float = 0.5) -> np.ndarray:
    """Coefficients [N^3][5][b] of a synthetic turbulent state of the
    five-variable system: rho = 1, m = v from ``turbulent_velocity`` with rms
    speed mach * sqrt(gamma p0), e = p0/(gamma-1) + v_rms^2/2 in the cell mean
    (higher modes of e zero): mean pressure p0, with the local kinetic energy
    taken out of it point by point."""
    c0 = float(np.sqrt(gamma * p0))
    v = turbulent_velocity(N, k, seed, mach, zeta, c0)
    u = np.zeros((N ** 3, 5, v.shape[2]))
    u[:, 0, 0] = 1.0
    u[:, 1:4, :] = v
    vrms2 = (v[:, :, 0] ** 2).sum(axis=1).mean()
    u[:, 4, 0] = p0 / (gamma - 1.0) + 0.5 * vrms2
    return u


def fourier_coeffs(N: int, k: int, kvec) -> np.ndarray:
    """Exact modal coefficients [N^3][b] (complex) of exp(2 pi i kvec . x)."""
    ijl = mode_degrees(k)
    fx = _axis_factors(N, k, int(kvec[0]))
    fy = _axis_factors(N, k, int(kvec[1]))
    fz = _axis_factors(N, k, int(kvec[2]))
    # cell (iz, iy, ix) -> index (iz*N + iy)*N + ix
    c = (fz[:, None, None, ijl[:, 2]] * fy[None, :, None, ijl[:, 1]] * fx[None, None, :, ijl[:, 0]])
    return c.reshape(N ** 3, len(ijl))


def sound_wave(N: int, k: int, eps: float = 1e-6, cs: float = 1.0, kvec=(1, 0, 0), v0=(0.0, 0.0, 0.0),
               t: float = 0.0) -> np.ndarray:
    """Linear acoustic wave rho = 1 + eps sin(theta), v = v0 + eps cs khat sin(theta),
    theta = 2 pi (kvec.x) - 2 pi |kvec| (cs + khat.v0) t, projected exactly.

    The momentum m = rho v contains the product eps^2 sin^2 (a 2*kvec mode),
    which is included exactly."""
    kv = np.asarray(kvec, dtype=np.float64)
    kn = np.sqrt((kv ** 2).sum())
    khat = kv / kn
    v0 = np.asarray(v0, dtype=np.float64)
    w = 2 * np.pi * kn * (cs + khat @ v0)
    ph = np.exp(-1j * w * t)
    e1 = fourier_coeffs(N, k, kvec) * ph          # exp(i theta)
    e2 = fourier_coeffs(N, k, 2 * kv.astype(int)) * ph * ph   # exp(2 i theta)
    b = nmodes(k)
    sin1 = e1.imag
    # sin^2 = (1 - cos 2theta)/2
    one = np.zeros((N ** 3, b))
    one[:, 0] = 1.0
    sin2 = 0.5 * (one - e2.real)
    u = np.zeros((N ** 3, 4, b))
    u[:, 0] = one + eps * sin1
    for i in range(3):
        # m_i = (1 + eps s)(v0_i + eps cs khat_i s)
        u[:, 1 + i] = v0[i] * one + eps * (v0[i] + cs * khat[i]) * sin1 + eps * eps * cs * khat[i] * sin2
    return u


def turbulent_velocity(N: int, k: int, seed: int, mach: float, zeta: float = 0.5, cs: float = 1.0,
                       kmin: float = 2.0, kmax: float | None = None, slope: float = -2.0) -> np.ndarray:
    """Coefficients [N^3][3][b] of a Gaussian random velocity field with shell
    spectrum E(k) ~ k^slope for kmin <= |k| <= kmax (integer wave vectors on
    the N^3 lattice), Helmholtz-mixed with solenoidal weight zeta, scaled so
    that the rms cell-mean speed is mach * cs.  Exact per-cell coefficients
    through an inverse FFT per Legendre mode."""
    if kmax is None:
        kmax = N / 4
    rng = np.random.default_rng(seed)
    kk = np.fft.fftfreq(N, d=1.0 / N)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    band = (K >= kmin) & (K <= kmax)
    amp = np.zeros_like(K)
    amp[band] = K[band] ** ((slope - 2.0) / 2.0)
    A = (rng.standard_normal((3,) + K.shape) + 1j * rng.standard_normal((3,) + K.shape)) * amp
    Ks = np.where(K > 0, K, 1.0)
    kh = np.stack([KX / Ks, KY / Ks, KZ / Ks])
    kdotA = (kh * A).sum(axis=0)
    comp = kh * kdotA
    A = zeta * (A - comp) + (1.0 - zeta) * comp
    ijl = mode_degrees(k)
    b = len(ijl)
    h = 1.0 / N
    m = np.arange(k + 1)

    def g(kap):
        return np.sqrt(2 * m + 1)[None, :] * (1j ** m)[None, :] * spherical_jn(m[None, :], np.pi * kap[:, None] * h)

    gx, gy, gz = g(KX.ravel()), g(KY.ravel()), g(KZ.ravel())
    out = np.zeros((N ** 3, 3, b))
    # field(x_c) = Re sum_k A_k prod_d g_{m_d}(k_d) exp(2 pi i k.x_c); x_c = (i + 1/2) h
    shift = np.exp(1j * np.pi * (KX + KY + KZ) / N)
    for l, (i, j, lz) in enumerate(ijl):
        G = (gx[:, i] * gy[:, j] * gz[:, lz]).reshape(K.shape) * shift
        for c in range(3):
            f = np.fft.ifftn(A[c] * G) * N ** 3
            out[:, c, l] = f.real.reshape(-1)
    rms = np.sqrt((out[:, :, 0] ** 2).sum(axis=1).mean())
    out *= mach * cs / rms
    return out


def turbulent_state_device(N: int, k: int, seed: int, mach: float, zeta: float = 0.5, cs: float = 1.0,
                           device="cuda", dtype=None, kmin: float = 2.0, kmax: float | None = None,
                           slope: float = -2.0):
    """``turbulent_state`` built with torch on ``device`` (the inverse FFTs run
    there; meshes of 256^3 and more): the same random draws (numpy, same seed)
    and the same recipe, returned as a torch tensor [N^3][4][b] of ``dtype``
    (float32 by default)."""
    import torch
    dtype = torch.float32 if dtype is None else dtype
    if kmax is None:
        kmax = N / 4
    rng = np.random.default_rng(seed)
    kk = np.fft.fftfreq(N, d=1.0 / N)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    band = (K >= kmin) & (K <= kmax)
    amp = np.zeros_like(K)
    amp[band] = K[band] ** ((slope - 2.0) / 2.0)
    del band
    # the draws in the numpy recipe's order: real parts of all three components, then imaginary
    re = rng.standard_normal((3,) + K.shape)
    im = rng.standard_normal((3,) + K.shape)
    A = torch.complex(torch.from_numpy(re), torch.from_numpy(im)).to(device) * torch.from_numpy(amp).to(device)
    del re, im
    Kd = torch.from_numpy(K).to(device)
    Ks = torch.where(Kd > 0, Kd, torch.ones_like(Kd))
    kx, ky, kz = (torch.from_numpy(x).to(device) for x in (KX, KY, KZ))
    del KX, KY, KZ, K
    kh = torch.stack([kx / Ks, ky / Ks, kz / Ks])
    del kx, ky, kz, Ks
    kdotA = (kh * A).sum(dim=0)
    comp = kh * kdotA
    A = zeta * (A - comp) + (1.0 - zeta) * comp
    del kh, kdotA, comp
    ijl = mode_degrees(k)
    b = len(ijl)
    h = 1.0 / N
    m = np.arange(k + 1)
    # per-axis factors sqrt(2m+1) i^m j_m(pi kappa h) and the half-cell shift exp(i pi kappa / N)
    g1 = np.sqrt(2 * m + 1)[None, :] * (1j ** m)[None, :] * spherical_jn(m[None, :], np.pi * kk[:, None] * h)
    g1 = g1 * np.exp(1j * np.pi * kk / N)[:, None]
    g = torch.from_numpy(g1).to(device)
    u = torch.zeros(N ** 3, 4, b, dtype=dtype, device=device)
    u[:, 0, 0] = 1.0
    for l, (i, j, lz) in enumerate(ijl):
        G = g[:, lz][:, None, None] * g[:, j][None, :, None] * g[:, i][None, None, :]
        for c in range(3):
            f = torch.fft.ifftn(A[c] * G) * (N ** 3)
            u[:, 1 + c, l] = f.real.reshape(-1).to(dtype)
    rms = torch.sqrt((u[:, 1:, 0].double() ** 2).sum(dim=1).mean())
    u[:, 1:, :] *= float(mach * cs / rms)
    return u


def turbulent_state(N: int, k: int, seed: int, mach: float, zeta: float = 0.5, cs: float = 1.0) -> np.ndarray:
    """rho = 1 and m = v from ``turbulent_velocity``: the start of a relaxation run."""
    v = turbulent_velocity(N, k, seed, mach, zeta, cs)
    u = np.zeros((N ** 3, 4, v.shape[2]))
    u[:, 0, 0] = 1.0
    u[:, 1:, :] = v
    return u


def uniform_state(N: int, k: int, rho: float = 1.0, v=(0.0, 0.0, 0.0)) -> np.ndarray:
    u = np.zeros((N ** 3, 4, nmodes(k)))
    u[:, 0, 0] = rho
    for i in range(3):
        u[:, 1 + i, 0] = rho * v[i]
    return u


def mlp_init(D: int, seed: int, H: int = 64) -> np.ndarray:
    """Seeded Kaiming-uniform parameters of the learned sensor's network in the
    library's flat layout (W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [H], b3):
    weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)), biases zero.  FP32."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (H, D)) * np.sqrt(6.0 / D)
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    W3 = rng.uniform(-1, 1, H) * np.sqrt(6.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, np.zeros(1)]).astype(np.float32)
