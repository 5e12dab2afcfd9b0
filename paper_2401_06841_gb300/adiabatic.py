"""Python front end of the adiabatic system of libdg (include/dg.h, dg_adi_*):
owns the device buffers (torch tensors) and the stream, forwards every call
to the C ABI.  No arithmetic of the method happens here."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as B
from .solver import nmodes


class AdiabaticSolver:
    """Five-variable DG context (rho, m_x, m_y, m_z, e) on one GPU.

    N cells per axis, degree k (1..3), adiabatic index gamma; precision 'f64'
    or 'f32'; av 'off' | 'vnr'."""

    def __init__(self, N: int, k: int, gamma: float = 1.4, precision: str = "f32", rk_stages: int | None = None,
                 cfl: float = 0.3, av: str = "vnr", alpha: float = 2.0, beta: float = 0.2, floor: float = 1e-3,
                 device: str | int = "cuda", riemann: str = "rusanov", bc=("periodic",) * 3,
                 inflow=(1.0, 0.0, 0.0, 0.0, 1.0)):
        self.L = B.lib()
        self.h = None
        self.N, self.k, self.gamma = N, k, gamma
        self.b = nmodes(k)
        self.ncell = N ** 3
        self.prec = {"f64": B.PREC_F64, "f32": B.PREC_F32}[precision]
        self.dtype = torch.float64 if self.prec == B.PREC_F64 else torch.float32
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.Stream(device=self.device)
        if rk_stages is None:
            rk_stages = 2 if k == 1 else 3
        self.mesh = B.Mesh((C.c_int32 * 3)(N, N, N), (C.c_double * 3)(1.0, 1.0, 1.0))
        self.nu = B.NuParams({"off": B.AV_OFF, "vnr": B.AV_VNR}[av], alpha, beta, floor, 0.0, 0.0, 0)
        sb, pb, cb = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
        self._check(self.L.dg_adi_buffer_bytes(C.byref(self.mesh), k, self.prec, C.byref(sb), C.byref(pb),
                                               C.byref(cb)), None)
        with torch.cuda.device(self.device):
            self.regs = [torch.zeros(self.ncell, 5, self.b, dtype=self.dtype, device=self.device) for _ in range(3)]
            self.prim = torch.zeros(self.ncell, 4, self.b, dtype=self.dtype, device=self.device)
            self.scratch = torch.zeros(int(cb.value), dtype=torch.uint8, device=self.device)
        o = B.AdiOpts(self.prec, rk_stages, cfl, gamma, C.c_void_p(self.stream.cuda_stream),
                      (C.c_void_p * 3)(*[r.data_ptr() for r in self.regs]), self.prim.data_ptr(),
                      self.scratch.data_ptr(), int(cb.value), {"rusanov": 0, "hllc": 2}[riemann],
                      (C.c_int32 * 3)(*[{"periodic": 0, "outflow": 1, "reflect": 2, "inflow": 3}[x] for x in bc]),
                      (C.c_double * 5)(*inflow))
        torch.cuda.synchronize(self.device)
        h = C.c_void_p()
        self._check(self.L.dg_adi_init(C.byref(h), C.byref(self.mesh), k, C.byref(self.nu), C.byref(o)), None)
        self.h = h

    def _check(self, rc: int, h):
        if rc != 0:
            msg = self.L.dg_adi_last_error(h).decode() if h else ""
            raise B.DGError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.dg_adi_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _as_dev(self, x, shape):
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x))
        x = x.to(device=self.device, dtype=self.dtype).contiguous()
        assert tuple(x.shape) == shape, (tuple(x.shape), shape)
        return x

    def set_state(self, u):
        """u: [N^3, 5, b] (numpy or torch, host or device)."""
        if isinstance(u, np.ndarray):
            t = torch.from_numpy(np.ascontiguousarray(u.astype(np.float64 if self.prec == B.PREC_F64 else np.float32)))
            self._check(self.L.dg_adi_set_state(self.h, t.data_ptr(), 1), self.h)
        else:
            t = self._as_dev(u, (self.ncell, 5, self.b))
            torch.cuda.current_stream(self.device).synchronize()
            self._check(self.L.dg_adi_set_state(self.h, t.data_ptr(), 0), self.h)

    def get_state(self) -> torch.Tensor:
        out = torch.empty(self.ncell, 5, self.b, dtype=self.dtype, device=self.device)
        self._check(self.L.dg_adi_get_state(self.h, out.data_ptr(), 0), self.h)
        return out

    def project(self, u) -> torch.Tensor:
        u = self._as_dev(u, (self.ncell, 5, self.b))
        out = torch.empty(self.ncell, 4, self.b, dtype=self.dtype, device=self.device)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_adi_project(self.h, u.data_ptr(), out.data_ptr()), self.h)
        return out

    def rhs(self, u, dt_pimax: float = 0.0) -> torch.Tensor:
        u = self._as_dev(u, (self.ncell, 5, self.b))
        out = torch.empty_like(u)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_adi_rhs(self.h, u.data_ptr(), out.data_ptr(), dt_pimax), self.h)
        return out

    def step(self, nsteps: int = 1, fixed_dt: float = 0.0):
        t = C.c_double(0)
        dtl = C.c_double(0)
        self._check(self.L.dg_adi_step(self.h, nsteps, fixed_dt, C.byref(t), C.byref(dtl)), self.h)
        return t.value, dtl.value

    def set_forcing(self, mach: float, zeta: float = 0.5, seed: int = 0, kmin2: int = 1, kmax2: int = 9,
                    t_off: float = 0.0, on: bool = True, cs_ref: float = 1.0):
        f = B.Forcing(1 if on else 0, kmin2, kmax2, zeta, mach, seed, t_off)
        self._check(self.L.dg_adi_set_forcing(self.h, C.byref(f), cs_ref), self.h)

    def set_reset(self, cs: float):
        """cs > 0: restore the uniform temperature p = cs^2 rho after every step."""
        self._check(self.L.dg_adi_set_reset(self.h, cs), self.h)

    def energy_budget(self):
        """(injected, dissipated) energy since set_state."""
        out = (C.c_double * 2)()
        self._check(self.L.dg_adi_energy_budget(self.h, out), self.h)
        return out[0], out[1]

    def get_meta(self):
        m = B.AdiMeta()
        self._check(self.L.dg_adi_get_meta(self.h, C.byref(m)), self.h)
        return m

    def set_meta(self, m):
        self._check(self.L.dg_adi_set_meta(self.h, C.byref(m)), self.h)

    def totals(self) -> dict:
        out = (C.c_double * 8)()
        self._check(self.L.dg_adi_totals(self.h, out), self.h)
        names = ("mass", "mom_x", "mom_y", "mom_z", "energy", "ekin", "rho_min", "p_min")
        return {n: out[i] for i, n in enumerate(names)}
