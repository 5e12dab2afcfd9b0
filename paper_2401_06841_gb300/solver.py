"""Python front end of libdg: owns the device buffers (torch tensors) and the
stream, and forwards every call to the C ABI.  No arithmetic of the method
happens here."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as B


def nmodes(k: int) -> int:
    return (k + 1) * (k + 2) * (k + 3) // 6


class Solver:
    """DG solver context on one GPU.

    N cells per axis, degree k (1..3), sound speed cs; precision 'f64', 'f32'
    or 'x3'; av 'off' | 'vnr' | 'learned'; face flux riemann 'rusanov' | 'hll' | 'hllc';
    positivity 'scale' (rescale stage outputs) | 'repeat' (also repeat the step
    with troubled cells of u^n flattened, Sec. 3.1)."""

    def __init__(self, N: int, k: int, cs: float = 1.0, precision: str = "f32", rk_stages: int | None = None,
                 cfl: float = 0.3, av: str = "vnr", alpha: float = 2.0, beta: float = 0.2, rho_floor: float = 1e-3,
                 nu_gate: float = 0.0, device: str | int = "cuda", stream: torch.cuda.Stream | None = None,
                 riemann: str = "rusanov", diffusion: float = 0.0, fused_infer: bool = False,
                 x3_backend: str = "tcgen05", positivity: str = "scale"):
        self.L = B.lib()
        self.N, self.k, self.cs = N, k, cs
        self.b = nmodes(k)
        self.ncell = N ** 3
        self.prec = {"f64": B.PREC_F64, "f32": B.PREC_F32, "x3": B.PREC_X3}[precision]
        self.dtype = torch.float64 if self.prec == B.PREC_F64 else torch.float32
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        if rk_stages is None:
            rk_stages = 2 if k == 1 else 3
        self.rk = rk_stages
        av_mode = {"off": B.AV_OFF, "vnr": B.AV_VNR, "learned": B.AV_LEARNED}[av]
        self.mesh = B.Mesh((C.c_int32 * 3)(N, N, N), (C.c_double * 3)(1.0, 1.0, 1.0))
        self.nu = B.NuParams(av_mode, alpha, beta, rho_floor, nu_gate, diffusion, int(fused_infer))
        nb = C.c_size_t(0)
        self._check(self.L.dg_scratch_bytes(C.byref(self.mesh), k, C.byref(self.nu), C.byref(nb)), None)
        with torch.cuda.device(self.device):
            self.regs = [torch.zeros(self.ncell, 4, self.b, dtype=self.dtype, device=self.device) for _ in range(3)]
            vb = C.c_size_t(0)
            self._check(self.L.dg_vhat_bytes(C.byref(self.mesh), k, self.prec, C.byref(vb)), None)
            self.vhat = torch.zeros(int(vb.value), dtype=torch.uint8, device=self.device)
            self.ahat = torch.zeros(self.ncell, 3, self.b, dtype=self.dtype, device=self.device)
            self.scratch = torch.zeros(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        base = self.scratch.data_ptr()
        off = (-base) % 256
        opts = B.Opts(self.prec, rk_stages, cfl, C.c_void_p(self.stream.cuda_stream),
                      (C.c_void_p * 3)(*[r.data_ptr() for r in self.regs]), self.vhat.data_ptr(),
                      self.ahat.data_ptr(), base + off, int(nb.value), B.RIEMANN[riemann],
                      {"tcgen05": 0, "mma": 1}[x3_backend], {"scale": 0, "repeat": 1}[positivity])
        torch.cuda.synchronize(self.device)
        h = C.c_void_p(0)
        rc = self.L.dg_init(C.byref(h), C.byref(self.mesh), k, cs, C.byref(self.nu), C.byref(opts))
        if rc != 0:
            raise B.DGError(rc, "dg_init failed")
        self.h = h

    # ------------------------------------------------------------------
    def _check(self, rc: int, h):
        if rc != 0:
            msg = self.L.dg_last_error(h).decode() if h else ""
            raise B.DGError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.dg_free(self.h)
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

    def sync(self):
        self.stream.synchronize()

    # ------------------------------------------------------------------
    def set_state(self, u):
        """u: [N^3, 4, b] array (numpy or torch, host or device)."""
        if isinstance(u, np.ndarray):
            t = torch.from_numpy(np.ascontiguousarray(u.astype(
                np.float64 if self.prec == B.PREC_F64 else np.float32)))
            self._check(self.L.dg_set_state(self.h, t.data_ptr(), 1), self.h)
        else:
            t = self._as_dev(u, (self.ncell, 4, self.b))
            torch.cuda.current_stream(self.device).synchronize()
            self._check(self.L.dg_set_state(self.h, t.data_ptr(), 0), self.h)

    def get_state(self) -> torch.Tensor:
        out = torch.empty(self.ncell, 4, self.b, dtype=self.dtype, device=self.device)
        self._check(self.L.dg_get_state(self.h, out.data_ptr(), 0), self.h)
        return out

    def rhs(self, u, ahat=None, dt_pimax: float = 0.0) -> torch.Tensor:
        u = self._as_dev(u, (self.ncell, 4, self.b))
        a = None if ahat is None else self._as_dev(ahat, (self.ncell, 3, self.b))
        out = torch.empty_like(u)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_rhs(self.h, u.data_ptr(), None if a is None else a.data_ptr(), out.data_ptr(),
                                  dt_pimax), self.h)
        return out

    def project_velocity(self, u) -> torch.Tensor:
        u = self._as_dev(u, (self.ncell, 4, self.b))
        out = torch.empty(self.ncell, 3, self.b, dtype=self.dtype, device=self.device)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_project_velocity(self.h, u.data_ptr(), out.data_ptr()), self.h)
        return out

    def step(self, nsteps: int = 1, fixed_dt: float = 0.0):
        t = C.c_double(0)
        dtl = C.c_double(0)
        self._check(self.L.dg_step(self.h, nsteps, fixed_dt, C.byref(t), C.byref(dtl)), self.h)
        return t.value, dtl.value

    def set_forcing(self, mach: float, zeta: float = 0.5, seed: int = 0, kmin2: int = 1, kmax2: int = 9,
                    t_off: float = 0.0, on: bool = True):
        f = B.Forcing(1 if on else 0, kmin2, kmax2, zeta, mach, seed, t_off)
        self._check(self.L.dg_set_forcing(self.h, C.byref(f)), self.h)

    def set_forcing_coeffs(self, ahat):
        if ahat is None:
            self._check(self.L.dg_set_forcing_coeffs(self.h, None, 0), self.h)
            return
        a = self._as_dev(ahat, (self.ncell, 3, self.b))
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_set_forcing_coeffs(self.h, a.data_ptr(), 0), self.h)

    def forcing_from_modes(self, kvec, amp) -> torch.Tensor:
        kv = np.ascontiguousarray(kvec, dtype=np.int32)
        am = np.ascontiguousarray(amp, dtype=np.float64)
        self._check(self.L.dg_forcing_from_modes(self.h, len(kv), kv.ctypes.data, am.ctypes.data), self.h)
        return self.ahat.clone()

    def diagnostics(self, dt_pimax: float = 0.0) -> dict:
        d = B.Diag()
        self._check(self.L.dg_diagnostics(self.h, dt_pimax, C.byref(d)), self.h)
        return {"mass": d.mass, "mom_x": d.mom[0], "mom_y": d.mom[1], "mom_z": d.mom[2], "ekin": d.ekin,
                "mach": d.mach, "mach_rho": d.mach_rho, "rho_min": d.rho_min, "rho_max": d.rho_max,
                "av_frac": d.av_frac, "inj_power": d.inj_power, "max_speed": d.max_speed, "av_work": d.av_work,
                "status": d.status, "t": d.t, "steps": d.steps}

    def l1_density(self, uA, uB) -> float:
        a = self._as_dev(uA, (self.ncell, 4, self.b))
        b = self._as_dev(uB, (self.ncell, 4, self.b))
        out = C.c_double(0)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_l1_density(self.h, a.data_ptr(), b.data_ptr(), C.byref(out)), self.h)
        return out.value

    def get_meta(self) -> B.Meta:
        m = B.Meta()
        self._check(self.L.dg_get_meta(self.h, C.byref(m)), self.h)
        return m

    def set_meta(self, m: B.Meta):
        self._check(self.L.dg_set_meta(self.h, C.byref(m)), self.h)

    def profile(self, enable: bool = True):
        self._check(self.L.dg_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self) -> dict:
        p = B.Prof()
        self._check(self.L.dg_profile_read(self.h, C.byref(p)), self.h)
        return {f: getattr(p, f) for f, _ in B.Prof._fields_}

    # ---- learned viscosity sensor ------------------------------------------
    def av_param_count(self) -> int:
        n = C.c_int64(0)
        self._check(self.L.dg_av_param_count(self.h, C.byref(n)), self.h)
        return n.value

    def set_av_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        self._check(self.L.dg_set_av_weights(self.h, w.ctypes.data, w.size), self.h)

    def get_av_weights(self) -> np.ndarray:
        w = np.zeros(self.av_param_count(), dtype=np.float32)
        self._check(self.L.dg_get_av_weights(self.h, w.ctypes.data, w.size), self.h)
        return w

    def generate_pairs(self, dt_pimax: float = 0.0):
        D = 2 * self.b
        x = torch.empty(self.ncell, D, dtype=torch.float32, device=self.device)
        y = torch.empty(self.ncell, dtype=torch.float32, device=self.device)
        n = C.c_int64(0)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_generate_pairs(self.h, dt_pimax, x.data_ptr(), y.data_ptr(), self.ncell, C.byref(n)),
                    self.h)
        return x, y

    # ------------------------------------------------------------------
    # turbulence statistics of the current state
    def density_pdf(self, lo: float = -2.0, hi: float = 2.0, nbins: int = 200) -> np.ndarray:
        """Volume fractions of log10(rho/rho_mean) in nbins equal bins on [lo, hi)."""
        h = np.zeros(nbins)
        self._check(self.L.dg_density_pdf(self.h, lo, hi, nbins, h.ctypes.data), self.h)
        return h

    def structure_function(self, nbins: int = 100, npairs: int = 100000, seed: int = 0):
        """(l, v(l)): second-order velocity structure function on logarithmic bins."""
        l = np.zeros(nbins)
        v = np.zeros(nbins)
        self._check(self.L.dg_structure_function(self.h, nbins, npairs, seed, l.ctypes.data, v.ctypes.data), self.h)
        return l, v

    def power_spectrum(self, nbins: int = 2000):
        """(mean |kappa|, summed power, mode count) per logarithmic |kappa| shell of
        the velocity on the (k+1)N grid."""
        nb = C.c_size_t(0)
        self._check(self.L.dg_analysis_bytes(C.byref(self.mesh), self.k, C.byref(nb)), None)
        work = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        base = work.data_ptr()
        off = (-base) % 256
        km = np.zeros(nbins)
        pw = np.zeros(nbins)
        cnt = np.zeros(nbins, dtype=np.int64)
        torch.cuda.synchronize(self.device)
        self._check(self.L.dg_power_spectrum(self.h, base + off, int(nb.value), nbins, km.ctypes.data,
                                             pw.ctypes.data, cnt.ctypes.data), self.h)
        del work
        return km, pw, cnt

    def mlp_train(self, x, y, epochs: int = 10, batch: int = 4096, lr: float = 1e-3) -> float:
        x = torch.as_tensor(x, dtype=torch.float32, device=self.device).contiguous()
        y = torch.as_tensor(y, dtype=torch.float32, device=self.device).contiguous()
        o = B.TrainOpts(lr, 0.9, 0.999, 1e-8, batch, epochs)
        loss = C.c_double(0)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_mlp_train(self.h, x.data_ptr(), y.data_ptr(), len(y), C.byref(o), C.byref(loss)), self.h)
        return loss.value

    def mlp_grad(self, x, y):
        x = torch.as_tensor(x, dtype=torch.float32, device=self.device).contiguous()
        y = torch.as_tensor(y, dtype=torch.float32, device=self.device).contiguous()
        g = torch.empty(self.av_param_count(), dtype=torch.float32, device=self.device)
        loss = C.c_double(0)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_mlp_grad(self.h, x.data_ptr(), y.data_ptr(), len(y), g.data_ptr(), C.byref(loss)),
                    self.h)
        return loss.value, g

    def mlp_forward(self, x):
        x = torch.as_tensor(x, dtype=torch.float32, device=self.device).contiguous()
        y = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.L.dg_mlp_forward(self.h, x.data_ptr(), x.shape[0], y.data_ptr()), self.h)
        return y

    def av_nu(self):
        nu = torch.empty(self.ncell, dtype=torch.float32, device=self.device)
        self._check(self.L.dg_av_nu(self.h, nu.data_ptr()), self.h)
        return nu

    def av_nu_carried(self):
        """The coefficient the last learned step evaluated for the current state."""
        nu = torch.empty(self.ncell, dtype=torch.float32, device=self.device)
        self._check(self.L.dg_av_nu_carried(self.h, nu.data_ptr()), self.h)
        return nu
