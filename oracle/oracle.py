"""ctypes wrapper of the FP64 CPU oracle (``dg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA library and its Python
binding never import this module.

Every array is a C-contiguous float64 numpy array in the cell-major layout
``u[cell][var][mode]`` with cell = (iz*N + iy)*N + ix.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_LIMITED = 1
ORC_FAIL = 2
NDIAG = 13
DIAG_NAMES = ("mass", "mom_x", "mom_y", "mom_z", "ekin", "mach", "mach_rho", "rho_min", "rho_max",
              "av_frac", "inj_power", "max_speed", "av_work")


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C compiler (plain C11, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dg_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(C.Structure):
    _fields_ = [("N", C.c_int32), ("k", C.c_int32), ("cs", C.c_double), ("av_mode", C.c_int32),
                ("alpha", C.c_double), ("beta", C.c_double), ("rho_floor", C.c_double), ("cfl", C.c_double),
                ("rk_stages", C.c_int32), ("riemann", C.c_int32), ("eps_diff", C.c_double),
                ("pos_mode", C.c_int32), ("bc", C.c_int32 * 3), ("inflow", C.c_double * 5)]


RIEMANN = {"rusanov": 0, "hll": 1, "hllc": 2}
POSITIVITY = {"scale": 0, "repeat": 1}
BC = {"periodic": 0, "outflow": 1, "reflect": 2, "inflow": 3}
REPEAT_SPEED = 1.5
ST_LIMITED, ST_FAIL, ST_REPEATED = 1, 2, 4
MARK_NEGATIVE, MARK_FAST = 1, 2


MAX_MODES = 512


class OU(C.Structure):
    _fields_ = [("nmodes", C.c_int32), ("kvec", C.c_int32 * 3 * MAX_MODES),
                ("x", C.c_double * 2 * 3 * MAX_MODES),
                ("zeta", C.c_double), ("sigma", C.c_double), ("tc", C.c_double), ("dt_drive", C.c_double),
                ("s", C.c_double), ("f", C.c_double), ("t_next", C.c_double), ("t_off", C.c_double),
                ("rng", C.c_uint64), ("have_spare", C.c_int32), ("spare", C.c_double), ("on", C.c_int32),
                ("dirty", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        _lib.orc_dt.restype = C.c_double
        _lib.orc_vnr.restype = C.c_double
        _lib.orc_legendre.restype = C.c_double
        _lib.orc_legendre_deriv.restype = C.c_double
        _lib.orc_l1_density.restype = C.c_double
        _lib.orc_splitmix64.restype = C.c_uint64
        _lib.orc_legendre.argtypes = [C.c_int, C.c_double]
        _lib.orc_legendre_deriv.argtypes = [C.c_int, C.c_double]
        _lib.orc_vnr.argtypes = [C.POINTER(Cfg), C.c_double, C.c_double, C.c_double]
        _lib.orc_rusanov.argtypes = [C.c_double, C.c_int, d, d, d]
        _lib.orc_riemann.argtypes = [C.c_int, C.c_double, C.c_int, d, d, d]
        _lib.orc_recover_dn.restype = C.c_double
        _lib.orc_recover_dn.argtypes = [C.c_int, d, d]
        _lib.orc_diffusion_rhs.argtypes = [C.POINTER(Cfg), d, d]
        _lib.orc_density_pdf.argtypes = [C.POINTER(Cfg), d, C.c_double, C.c_double, C.c_int, d]
        _lib.orc_structure_function.argtypes = [C.POINTER(Cfg), d, C.c_int, C.c_int64, C.c_uint64, d, d]
        _lib.orc_sample_velocity.argtypes = [C.POINTER(Cfg), d, d]
        _lib.orc_ou_init.argtypes = [C.POINTER(OU), C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_uint64, C.c_double]
        _lib.orc_rhs.argtypes = [C.POINTER(Cfg), d, d, C.c_double, d]
        _lib.orc_step.argtypes = [C.POINTER(Cfg), d, d, C.c_double]
        u8 = C.POINTER(C.c_uint8)
        _lib.orc_step_flags.argtypes = [C.POINTER(Cfg), d, d, C.c_double, C.c_double, u8]
        _lib.orc_speed_bound.restype = C.c_double
        _lib.orc_speed_bound.argtypes = [C.POINTER(Cfg), d]
        _lib.orc_step_repeat.argtypes = [C.POINTER(Cfg), d, d, C.c_double, d, C.POINTER(C.c_int), u8]
        _lib.orc_run.argtypes = [C.POINTER(Cfg), d, C.POINTER(OU), C.c_int, d, C.c_int, d, d]
        _lib.orc_diagnostics.argtypes = [C.POINTER(Cfg), d, d, C.c_double, d]
        _lib.orc_forcing_project.argtypes = [C.POINTER(Cfg), C.c_int, C.POINTER(C.c_int32), d, d]
        _lib.orc_rhs_nu.argtypes = [C.POINTER(Cfg), d, d, C.c_double, d, d]
        _lib.orc_rhs_local.argtypes = [C.POINTER(Cfg), d, d, d, C.c_double, d, C.c_int64, d]
        _lib.orc_adi_flux.argtypes = [C.c_double, C.c_int, d, d]
        _lib.orc_adi_rusanov.argtypes = [C.c_double, C.c_int, d, d, d]
        _lib.orc_adi_hllc.argtypes = [C.c_double, C.c_int, d, d, d]
        _lib.orc_adi_vnr.restype = C.c_double
        _lib.orc_adi_vnr.argtypes = [C.POINTER(Cfg), C.c_double, C.c_double, C.c_double, C.c_double]
        _lib.orc_adi_project.argtypes = [C.POINTER(Cfg), C.c_double, d, d]
        _lib.orc_adi_rhs.argtypes = [C.POINTER(Cfg), C.c_double, d, C.c_double, d]
        _lib.orc_adi_dt.restype = C.c_double
        _lib.orc_adi_dt.argtypes = [C.POINTER(Cfg), C.c_double, d]
        _lib.orc_adi_limit.argtypes = [C.POINTER(Cfg), C.c_double, d]
        _lib.orc_adi_step.argtypes = [C.POINTER(Cfg), C.c_double, d, C.c_double]
        _lib.orc_adi_run.argtypes = [C.POINTER(Cfg), C.c_double, d, C.c_int, C.c_double, d, d]
        _lib.orc_adi_rhs_forced.argtypes = [C.POINTER(Cfg), C.c_double, d, d, C.c_double, d, d]
        _lib.orc_adi_step_forced.argtypes = [C.POINTER(Cfg), C.c_double, d, d, C.c_double, d]
        _lib.orc_adi_reset.restype = C.c_double
        _lib.orc_adi_reset.argtypes = [C.POINTER(Cfg), C.c_double, C.c_double, d]
        _lib.orc_adi_run_driven.argtypes = [C.POINTER(Cfg), C.c_double, C.c_double, d, C.POINTER(OU), C.c_int, d,
                                            C.c_int, C.c_double, d, d, d, d]
        _lib.orc_av_features.argtypes = [C.POINTER(Cfg), d, C.c_double, d, d]
        _lib.orc_pi_nu.restype = C.c_double
        _lib.orc_pi_nu.argtypes = [C.POINTER(Cfg), C.c_double, C.c_double, C.c_double, C.c_double]
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (n > 0 sets it); returns the number in use."""
    return lib().orc_set_threads(int(n))


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def nmodes(k: int) -> int:
    return (k + 1) * (k + 2) * (k + 3) // 6


def mode_list(k: int) -> np.ndarray:
    b = nmodes(k)
    out = np.zeros((b, 3), dtype=np.int32)
    lib().orc_mode_list(C.c_int(k), out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


def gauss(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss(C.c_int(n), _p(x), _p(w))
    return x, w


def legendre(m: int, x: float) -> float:
    return lib().orc_legendre(m, x)


def legendre_deriv(m: int, x: float) -> float:
    return lib().orc_legendre_deriv(m, x)


def make_cfg(N, k, cs=1.0, av_mode=1, alpha=2.0, beta=0.2, rho_floor=1e-3, cfl=0.3, rk_stages=None,
             riemann="rusanov", eps_diff=0.0, positivity="scale", bc=("periodic",) * 3,
             inflow=(1.0, 0.0, 0.0, 0.0, 1.0)) -> Cfg:
    """bc, inflow: boundaries of the adiabatic system per axis ('periodic',
    'outflow', 'reflect', 'inflow' with the state inflow = (rho, v, p) at the
    lower face); the isothermal system is periodic."""
    if rk_stages is None:
        rk_stages = 2 if k == 1 else 3
    return Cfg(N, k, cs, av_mode, alpha, beta, rho_floor, cfl, rk_stages, RIEMANN[riemann], eps_diff,
               POSITIVITY[positivity], (C.c_int32 * 3)(*[BC[x] for x in bc]), (C.c_double * 5)(*inflow))


def _shape(cfg, nvar=4):
    return (cfg.N ** 3, nvar, nmodes(cfg.k))


def dt(cfg: Cfg, u: np.ndarray) -> float:
    return lib().orc_dt(C.byref(cfg), _p(u))


def project_velocity(cfg: Cfg, u: np.ndarray) -> np.ndarray:
    out = np.zeros(_shape(cfg, 3))
    lib().orc_project_velocity(C.byref(cfg), _p(u), _p(out))
    return out


def forcing_mean(cfg: Cfg, u: np.ndarray, ahat: np.ndarray) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_forcing_mean(C.byref(cfg), _p(u), _p(ahat), _p(out))
    return out


def vnr(cfg: Cfg, rho: float, divv: float, dt_: float) -> float:
    return lib().orc_vnr(C.byref(cfg), rho, divv, dt_)


def rusanov(cs: float, d: int, WL, WR) -> np.ndarray:
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(4)
    lib().orc_rusanov(cs, d, _p(WL), _p(WR), _p(F))
    return F


def riemann(solver: str, cs: float, d: int, WL, WR) -> np.ndarray:
    """Face flux along +e_d of the named solver ("rusanov", "hll", "hllc")."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(4)
    lib().orc_riemann(RIEMANN[solver], cs, d, _p(WL), _p(WR), _p(F))
    return F


def recover_dn(K: int, cL, cR) -> float:
    """d/ds at the face of the degree-2K+1 recovery of two cells' K+1 coefficients (s in half cells)."""
    cL = np.ascontiguousarray(cL, dtype=np.float64)
    cR = np.ascontiguousarray(cR, dtype=np.float64)
    return lib().orc_recover_dn(K, _p(cL), _p(cR))


def diffusion_rhs(cfg: Cfg, u: np.ndarray) -> np.ndarray:
    """The diffusion operator div(eps grad u) alone, in modal coefficients."""
    out = np.zeros(_shape(cfg))
    lib().orc_diffusion_rhs(C.byref(cfg), _p(u), _p(out))
    return out


def rhs(cfg: Cfg, u: np.ndarray, ahat: np.ndarray | None = None, dt_pimax: float = 0.0) -> np.ndarray:
    out = np.zeros(_shape(cfg))
    lib().orc_rhs(C.byref(cfg), _p(u), _p(ahat), dt_pimax, _p(out))
    return out


def rhs_nu(cfg: Cfg, u: np.ndarray, nu_cell: np.ndarray, ahat: np.ndarray | None = None,
           dt_pimax: float = 0.0) -> np.ndarray:
    """RHS with the per-cell viscous coefficient nu (learned-sensor mode)."""
    out = np.zeros(_shape(cfg))
    nu = np.ascontiguousarray(nu_cell, dtype=np.float64)
    lib().orc_rhs_nu(C.byref(cfg), _p(u), _p(ahat), dt_pimax, _p(nu), _p(out))
    return out


def neighbourhood(N: int, cells) -> np.ndarray:
    """[n][7] cell indices: each cell, then its periodic neighbours across the
    faces -x, +x, -y, +y, -z, +z (cell = (iz*N + iy)*N + ix)."""
    c = np.asarray(cells, dtype=np.int64)
    ix, iy, iz = c % N, (c // N) % N, c // (N * N)
    idx = lambda x, y, z: ((z % N) * N + (y % N)) * N + (x % N)  # noqa: E731
    return np.stack([c, idx(ix - 1, iy, iz), idx(ix + 1, iy, iz), idx(ix, iy - 1, iz), idx(ix, iy + 1, iz),
                     idx(ix, iy, iz - 1), idx(ix, iy, iz + 1)], axis=1)


def rhs_cells(cfg: Cfg, u: np.ndarray, cells, ahat: np.ndarray | None = None, abar=None, dt_pimax: float = 0.0,
              nu_cell: np.ndarray | None = None, base_N: int | None = None) -> np.ndarray:
    """RHS of the listed cells only (the same per-cell arithmetic as rhs), from
    each cell's face neighbourhood gathered out of u (any float array [N^3][4][b]).
    With ahat, abar is the mean acceleration of the whole field (forcing_mean).
    nu_cell: per-cell coefficients of the listed cells (learned mode) or None.
    base_N: u (and ahat) hold base_N^3 cells whose periodic tiling fills the
    N^3 mesh (N a multiple of base_N); cells index the N^3 mesh."""
    nb = neighbourhood(cfg.N, cells)
    if base_N is not None:
        assert cfg.N % base_N == 0
        x, y, z = nb % cfg.N, (nb // cfg.N) % cfg.N, nb // (cfg.N * cfg.N)
        nb = ((z % base_N) * base_N + (y % base_N)) * base_N + (x % base_N)
    patch = np.ascontiguousarray(np.asarray(u)[nb], dtype=np.float64)
    ac = None if ahat is None else np.ascontiguousarray(np.asarray(ahat)[nb[:, 0]], dtype=np.float64)
    ab = None if abar is None else np.ascontiguousarray(abar, dtype=np.float64)
    nu = None if nu_cell is None else np.ascontiguousarray(nu_cell, dtype=np.float64)
    out = np.zeros((len(nb), 4, patch.shape[-1]))
    rc = lib().orc_rhs_local(C.byref(cfg), _p(patch), _p(ac), _p(ab), dt_pimax, _p(nu), len(nb), _p(out))
    if rc != 0:
        raise ValueError("rhs_cells: not available with the diffusion operator")
    return out


def pi_nu(cfg: Cfg, rho: float, divv: float, nu: float, dt_: float) -> float:
    return lib().orc_pi_nu(C.byref(cfg), rho, divv, nu, dt_)


def av_features(cfg: Cfg, u: np.ndarray, dt_: float):
    """(x [cells][2b], y [cells]) inputs and targets of the learned sensor."""
    b = nmodes(cfg.k)
    x = np.zeros((cfg.N ** 3, 2 * b))
    y = np.zeros(cfg.N ** 3)
    lib().orc_av_features(C.byref(cfg), _p(u), dt_, _p(x), _p(y))
    return x, y


def limit(cfg: Cfg, u: np.ndarray) -> int:
    return lib().orc_limit(C.byref(cfg), _p(u))


def step(cfg: Cfg, u: np.ndarray, ahat: np.ndarray | None, dt_: float) -> int:
    """One SSP-RK step in place; returns the OR of the stage limiter statuses."""
    return lib().orc_step(C.byref(cfg), _p(u), _p(ahat), dt_)


def speed_bound(cfg: Cfg, u: np.ndarray) -> float:
    """S = max over cells and volume points of sum_d(|v_d| + cs)."""
    return lib().orc_speed_bound(C.byref(cfg), _p(u))


def step_flags(cfg: Cfg, u: np.ndarray, ahat: np.ndarray | None, dt_: float, vlim: float):
    """One SSP-RK step in place as ``step``; returns (status, flag[nc]) with the
    cells a stage troubled: MARK_NEGATIVE (rho < 0 at a point before the
    rescaling) | MARK_FAST (after it, a wave speed above vlim)."""
    flag = np.zeros(cfg.N ** 3, dtype=np.uint8)
    st = lib().orc_step_flags(C.byref(cfg), _p(u), _p(ahat), dt_, vlim,
                              flag.ctypes.data_as(C.POINTER(C.c_uint8)))
    return st, flag


def step_repeat(cfg: Cfg, u: np.ndarray, ahat: np.ndarray | None, fixed_dt: float = 0.0):
    """One step with positivity by repetition (Sec. 3.1), in place; returns
    (status or -1, dt used, attempts, level[nc] = how often each cell of u^n was
    scaled)."""
    dtu = C.c_double(0.0)
    att = C.c_int(0)
    level = np.zeros(cfg.N ** 3, dtype=np.uint8)
    st = lib().orc_step_repeat(C.byref(cfg), _p(u), _p(ahat), fixed_dt, C.byref(dtu), C.byref(att),
                               level.ctypes.data_as(C.POINTER(C.c_uint8)))
    return st, dtu.value, att.value, level


class Forcing:
    """Host OU driving state of the oracle (Sec. 4.2)."""

    def __init__(self, mach: float, zeta: float, seed: int, cs: float = 1.0, kmin2: int = 1, kmax2: int = 9,
                 t_off: float = 0.0):
        self.ou = OU()
        lib().orc_ou_init(C.byref(self.ou), kmin2, kmax2, zeta, mach, cs, 1.0, seed, t_off)

    @property
    def nmodes(self) -> int:
        return self.ou.nmodes

    def kvec(self) -> np.ndarray:
        return np.ctypeslib.as_array(self.ou.kvec)[: self.nmodes].copy()

    def x(self) -> np.ndarray:
        return np.ctypeslib.as_array(self.ou.x)[: self.nmodes].copy()

    def advance(self):
        lib().orc_ou_advance(C.byref(self.ou))

    def amplitudes(self) -> np.ndarray:
        amp = np.zeros((MAX_MODES, 3, 2))
        lib().orc_ou_amplitudes(C.byref(self.ou), _p(amp))
        return amp[: self.nmodes].copy()


def forcing_project(cfg: Cfg, kvec: np.ndarray, amp: np.ndarray) -> np.ndarray:
    kv = np.ascontiguousarray(kvec, dtype=np.int32)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    out = np.zeros(_shape(cfg, 3))
    lib().orc_forcing_project(C.byref(cfg), C.c_int(len(kv)), kv.ctypes.data_as(C.POINTER(C.c_int32)),
                              _p(amp), _p(out))
    return out


def run(cfg: Cfg, u: np.ndarray, nsteps: int, forcing: Forcing | None = None, t: float = 0.0,
        ahat: np.ndarray | None = None):
    """Advance ``u`` in place by ``nsteps`` steps (driving schedule + dt retry).

    Returns (rc, t, dt_last, ahat); ``ahat`` carries the current projected
    forcing between calls (pass it back in to continue a run)."""
    if ahat is None:
        ahat = np.zeros(_shape(cfg, 3))
    tt = C.c_double(t)
    dl = C.c_double(0.0)
    ou = forcing.ou if forcing is not None else OU()
    rc = lib().orc_run(C.byref(cfg), _p(u), C.byref(ou), 1 if forcing is not None else 0, _p(ahat), nsteps,
                       C.byref(tt), C.byref(dl))
    return rc, tt.value, dl.value, ahat


def diagnostics(cfg: Cfg, u: np.ndarray, ahat: np.ndarray | None = None, dt_: float = 0.0) -> dict:
    out = np.zeros(NDIAG)
    lib().orc_diagnostics(C.byref(cfg), _p(u), _p(ahat), dt_, _p(out))
    return dict(zip(DIAG_NAMES, out.tolist()))


def l1_density(cfg: Cfg, uA: np.ndarray, uB: np.ndarray) -> float:
    return lib().orc_l1_density(C.byref(cfg), _p(uA), _p(uB))


def density_pdf(cfg: Cfg, u: np.ndarray, lo: float, hi: float, nbins: int) -> np.ndarray:
    """Volume fractions of log10(rho/rho_mean) in nbins equal bins on [lo, hi)."""
    h = np.zeros(nbins)
    lib().orc_density_pdf(C.byref(cfg), _p(u), C.c_double(lo), C.c_double(hi), nbins, _p(h))
    return h


def structure_function(cfg: Cfg, u: np.ndarray, nbins: int, npairs: int, seed: int):
    """(l, v(l)) on nbins logarithmic bins (second-order velocity structure function)."""
    l = np.zeros(nbins)
    v = np.zeros(nbins)
    lib().orc_structure_function(C.byref(cfg), _p(u), nbins, C.c_int64(npairs), C.c_uint64(seed), _p(l), _p(v))
    return l, v


def sample_velocity(cfg: Cfg, u: np.ndarray) -> np.ndarray:
    """v on the (k+1)N regular grid at cell-interior points, shape [3][Ng][Ng][Ng] (z, y, x)."""
    Ng = (cfg.k + 1) * cfg.N
    out = np.zeros((3, Ng, Ng, Ng))
    lib().orc_sample_velocity(C.byref(cfg), _p(u), _p(out))
    return out


def power_spectrum(cfg: Cfg, u: np.ndarray, nbins: int):
    """Shell sums of the velocity power on the (k+1)N grid (Sec. 4.3):
    v_hat = FFT(v) / Ng^3 over integer wave vectors kappa; bins logarithmic in
    |kappa| with edges (sqrt(3) Ng/2)^(i/nbins), i = 0..nbins (the last edge
    included); kappa = 0 left out.  Returns (mean |kappa|, summed power
    sum_d |v_hat_d|^2, mode count) per bin; E(k) ~ power / bin width."""
    v = sample_velocity(cfg, u)
    Ng = v.shape[1]
    P = np.zeros((Ng, Ng, Ng))
    for d in range(3):
        P += np.abs(np.fft.fftn(v[d]) / Ng ** 3) ** 2
    f = np.fft.fftfreq(Ng, d=1.0 / Ng)
    KZ, KY, KX = np.meshgrid(f, f, f, indexing="ij")
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kmax = math.sqrt(3.0) * Ng / 2
    sel = K > 0
    idx = np.floor(np.log(K[sel]) / math.log(kmax) * nbins).astype(np.int64)
    idx = np.minimum(idx, nbins - 1)
    power = np.bincount(idx, weights=P[sel], minlength=nbins)
    count = np.bincount(idx, minlength=nbins)
    ksum = np.bincount(idx, weights=K[sel], minlength=nbins)
    kmean = np.where(count > 0, ksum / np.maximum(count, 1), 0.0)
    return kmean, power, count


def splitmix64(state: int, n: int) -> list[int]:
    s = C.c_uint64(state)
    return [lib().orc_splitmix64(C.byref(s)) for _ in range(n)]


# ---- adiabatic system: u [N^3][5][b] = (rho, m, e), primitives [N^3][4][b] = (v, p) ----
def adi_flux(gamma: float, d: int, U) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_adi_flux(gamma, d, _p(U), _p(F))
    return F


def adi_rusanov(gamma: float, d: int, WL, WR) -> np.ndarray:
    """Rusanov flux from primitive face states (rho, v_x, v_y, v_z, p)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_adi_rusanov(gamma, d, _p(WL), _p(WR), _p(F))
    return F


def adi_hllc(gamma: float, d: int, WL, WR) -> np.ndarray:
    """HLLC flux of the Euler equations from primitive face states (rho, v_x, v_y, v_z, p)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_adi_hllc(gamma, d, _p(WL), _p(WR), _p(F))
    return F


def adi_vnr(cfg: Cfg, rho: float, c: float, divv: float, dt_: float) -> float:
    return lib().orc_adi_vnr(C.byref(cfg), rho, c, divv, dt_)


def adi_project(cfg: Cfg, gamma: float, u: np.ndarray) -> np.ndarray:
    out = np.zeros((cfg.N ** 3, 4, nmodes(cfg.k)))
    lib().orc_adi_project(C.byref(cfg), gamma, _p(u), _p(out))
    return out


def adi_rhs(cfg: Cfg, gamma: float, u: np.ndarray, dt_pimax: float = 0.0) -> np.ndarray:
    out = np.zeros((cfg.N ** 3, 5, nmodes(cfg.k)))
    lib().orc_adi_rhs(C.byref(cfg), gamma, _p(u), dt_pimax, _p(out))
    return out


def adi_dt(cfg: Cfg, gamma: float, u: np.ndarray) -> float:
    return lib().orc_adi_dt(C.byref(cfg), gamma, _p(u))


def adi_limit(cfg: Cfg, gamma: float, u: np.ndarray) -> int:
    """Positivity of density and pressure, in place; returns the status bits."""
    return lib().orc_adi_limit(C.byref(cfg), gamma, _p(u))


def adi_step(cfg: Cfg, gamma: float, u: np.ndarray, dt_: float) -> int:
    return lib().orc_adi_step(C.byref(cfg), gamma, _p(u), dt_)


def adi_run(cfg: Cfg, gamma: float, u: np.ndarray, nsteps: int, fixed_dt: float = 0.0, t: float = 0.0):
    """Advance u in place; returns (rc, t, dt_last)."""
    tt = C.c_double(t)
    dl = C.c_double(0.0)
    rc = lib().orc_adi_run(C.byref(cfg), gamma, _p(u), nsteps, fixed_dt, C.byref(tt), C.byref(dl))
    return rc, tt.value, dl.value


def adi_rhs_forced(cfg: Cfg, gamma: float, u: np.ndarray, ahat: np.ndarray, dt_pimax: float = 0.0):
    """RHS with the driving a_h; returns (dudt, work integral of the energy source)."""
    out = np.zeros((cfg.N ** 3, 5, nmodes(cfg.k)))
    w = C.c_double(0.0)
    lib().orc_adi_rhs_forced(C.byref(cfg), gamma, _p(u), _p(ahat), dt_pimax, _p(out), C.byref(w))
    return out, w.value


def adi_reset(cfg: Cfg, gamma: float, cs: float, u: np.ndarray) -> float:
    """Isothermal reset of the thermal energy in place; returns the energy taken out."""
    return lib().orc_adi_reset(C.byref(cfg), gamma, cs, _p(u))


def adi_run_driven(cfg: Cfg, gamma: float, cs: float, u: np.ndarray, nsteps: int, forcing: Forcing | None = None,
                   fixed_dt: float = 0.0, t: float = 0.0, ahat: np.ndarray | None = None, budget=(0.0, 0.0)):
    """Driven adiabatic run with the isothermal reset (cs > 0); returns
    (rc, t, dt_last, ahat, (injected, dissipated))."""
    if ahat is None:
        ahat = np.zeros(_shape(cfg, 3))
    tt = C.c_double(t)
    dl = C.c_double(0.0)
    inj = C.c_double(budget[0])
    dis = C.c_double(budget[1])
    ou = forcing.ou if forcing is not None else OU()
    rc = lib().orc_adi_run_driven(C.byref(cfg), gamma, cs, _p(u), C.byref(ou), 1 if forcing is not None else 0,
                                  _p(ahat), nsteps, fixed_dt, C.byref(tt), C.byref(dl), C.byref(inj), C.byref(dis))
    return rc, tt.value, dl.value, ahat, (inj.value, dis.value)
