"""ctypes binding of libdg (include/dg.h): argument marshalling only.

Every step of the method runs in the CUDA library; torch supplies device
memory and the stream.  Importing this module fails loudly when libdg.so has
not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")

DG_OK, DG_EINVAL, DG_ECUDA, DG_ENOMEM, DG_EPOSITIVITY, DG_ENONFINITE, DG_ESTATE = range(7)
PREC_F64, PREC_F32, PREC_X3 = 0, 1, 2
AV_OFF, AV_VNR, AV_LEARNED = 0, 1, 2
RIEMANN = {"rusanov": 0, "hll": 1, "hllc": 2}
ST_LIMITED, ST_FAIL, ST_NONFINITE, ST_TIMEOUT, ST_REPEATED = 1, 2, 4, 8, 16
ERROR_NAMES = {DG_EINVAL: "DG_EINVAL", DG_ECUDA: "DG_ECUDA", DG_ENOMEM: "DG_ENOMEM",
               DG_EPOSITIVITY: "DG_EPOSITIVITY", DG_ENONFINITE: "DG_ENONFINITE", DG_ESTATE: "DG_ESTATE"}


class Mesh(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("L", C.c_double * 3)]


class NuParams(C.Structure):
    _fields_ = [("mode", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double), ("rho_floor", C.c_double),
                ("nu_gate", C.c_double), ("diffusion", C.c_double), ("fused_infer", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rk_stages", C.c_int32), ("cfl", C.c_double), ("stream", C.c_void_p),
                ("u", C.c_void_p * 3), ("vhat", C.c_void_p), ("ahat", C.c_void_p), ("scratch", C.c_void_p),
                ("scratch_bytes", C.c_size_t), ("riemann", C.c_int32), ("x3_backend", C.c_int32),
                ("positivity", C.c_int32)]


class AdiOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rk_stages", C.c_int32), ("cfl", C.c_double), ("gamma", C.c_double),
                ("stream", C.c_void_p), ("u", C.c_void_p * 3), ("prim", C.c_void_p), ("scratch", C.c_void_p),
                ("scratch_bytes", C.c_size_t), ("riemann", C.c_int32), ("bc", C.c_int32 * 3),
                ("inflow", C.c_double * 5)]


class Forcing(C.Structure):
    _fields_ = [("on", C.c_int32), ("kmin2", C.c_int32), ("kmax2", C.c_int32), ("zeta", C.c_double),
                ("mach", C.c_double), ("seed", C.c_uint64), ("t_off", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("mom", C.c_double * 3), ("ekin", C.c_double), ("mach", C.c_double),
                ("mach_rho", C.c_double), ("rho_min", C.c_double), ("rho_max", C.c_double),
                ("av_frac", C.c_double), ("inj_power", C.c_double), ("max_speed", C.c_double),
                ("av_work", C.c_double), ("status", C.c_uint32), ("t", C.c_double), ("steps", C.c_int64)]


class Meta(C.Structure):
    _fields_ = [("t", C.c_double), ("steps", C.c_int64), ("dt_last", C.c_double), ("forcing_on", C.c_int32),
                ("forcing_dirty", C.c_int32), ("t_next", C.c_double), ("rng", C.c_uint64),
                ("have_spare", C.c_int32), ("spare", C.c_double), ("nmodes", C.c_int32),
                ("x", C.c_double * 2 * 3 * 512)]


class AdiMeta(C.Structure):
    _fields_ = [("m", Meta), ("injected", C.c_double), ("dissipated", C.c_double)]


class TrainOpts(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("batch", C.c_int32), ("epochs", C.c_int32)]


class Prof(C.Structure):
    _fields_ = [("launches", C.c_int64), ("n_project", C.c_int64), ("n_rhs", C.c_int64), ("n_force", C.c_int64),
                ("n_other", C.c_int64), ("ms_project", C.c_double), ("ms_rhs", C.c_double),
                ("ms_force", C.c_double), ("ms_other", C.c_double), ("tiles_volume", C.c_int64),
                ("tiles_gated", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load libdg.so (built in-tree by paper_2401_06841_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdg.so is not built: run paper_2401_06841_gb300.build.build() "
                              "(nvcc, sm_103a); there is no fallback implementation")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.dg_scratch_bytes.argtypes = [C.POINTER(Mesh), i, C.POINTER(NuParams), C.POINTER(C.c_size_t)]
        L.dg_vhat_bytes.argtypes = [C.POINTER(Mesh), i, i, C.POINTER(C.c_size_t)]
        L.dg_init.argtypes = [C.POINTER(vp), C.POINTER(Mesh), i, d, C.POINTER(NuParams), C.POINTER(Opts)]
        L.dg_free.argtypes = [vp]
        L.dg_free.restype = None
        L.dg_last_error.argtypes = [vp]
        L.dg_last_error.restype = C.c_char_p
        L.dg_set_state.argtypes = [vp, vp, i]
        L.dg_get_state.argtypes = [vp, vp, i]
        L.dg_rhs.argtypes = [vp, vp, vp, vp, d]
        L.dg_project_velocity.argtypes = [vp, vp, vp]
        L.dg_step.argtypes = [vp, i, d, C.POINTER(d), C.POINTER(d)]
        L.dg_set_forcing.argtypes = [vp, C.POINTER(Forcing)]
        L.dg_set_forcing_coeffs.argtypes = [vp, vp, i]
        L.dg_forcing_from_modes.argtypes = [vp, i, vp, vp]
        L.dg_diagnostics.argtypes = [vp, d, C.POINTER(Diag)]
        L.dg_l1_density.argtypes = [vp, vp, vp, C.POINTER(d)]
        L.dg_get_meta.argtypes = [vp, C.POINTER(Meta)]
        L.dg_set_meta.argtypes = [vp, C.POINTER(Meta)]
        L.dg_av_param_count.argtypes = [vp, C.POINTER(C.c_int64)]
        L.dg_set_av_weights.argtypes = [vp, vp, C.c_size_t]
        L.dg_get_av_weights.argtypes = [vp, vp, C.c_size_t]
        L.dg_generate_pairs.argtypes = [vp, d, vp, vp, C.c_int64, C.POINTER(C.c_int64)]
        L.dg_mlp_train.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(TrainOpts), C.POINTER(d)]
        L.dg_mlp_grad.argtypes = [vp, vp, vp, C.c_int64, vp, C.POINTER(d)]
        L.dg_mlp_forward.argtypes = [vp, vp, C.c_int64, vp]
        L.dg_av_nu.argtypes = [vp, vp]
        L.dg_av_nu_carried.argtypes = [vp, vp]
        sz = C.POINTER(C.c_size_t)
        L.dg_adi_buffer_bytes.argtypes = [C.POINTER(Mesh), i, i, sz, sz, sz]
        L.dg_adi_init.argtypes = [C.POINTER(vp), C.POINTER(Mesh), i, C.POINTER(NuParams), C.POINTER(AdiOpts)]
        L.dg_adi_free.argtypes = [vp]
        L.dg_adi_free.restype = None
        L.dg_adi_last_error.argtypes = [vp]
        L.dg_adi_last_error.restype = C.c_char_p
        L.dg_adi_set_state.argtypes = [vp, vp, i]
        L.dg_adi_get_state.argtypes = [vp, vp, i]
        L.dg_adi_project.argtypes = [vp, vp, vp]
        L.dg_adi_rhs.argtypes = [vp, vp, vp, d]
        L.dg_adi_step.argtypes = [vp, i, d, C.POINTER(d), C.POINTER(d)]
        L.dg_adi_totals.argtypes = [vp, C.POINTER(d)]
        L.dg_adi_set_forcing.argtypes = [vp, C.POINTER(Forcing), d]
        L.dg_adi_set_reset.argtypes = [vp, d]
        L.dg_adi_energy_budget.argtypes = [vp, C.POINTER(d)]
        L.dg_adi_get_meta.argtypes = [vp, C.POINTER(AdiMeta)]
        L.dg_adi_set_meta.argtypes = [vp, C.POINTER(AdiMeta)]
        L.dg_rhs_noalloc.argtypes = [C.POINTER(Mesh), i, d, C.POINTER(NuParams), i, vp, vp, vp, d, vp]
        L.dg_profile.argtypes = [vp, i]
        L.dg_profile_read.argtypes = [vp, C.POINTER(Prof)]
        L.dg_density_pdf.argtypes = [vp, d, d, i, vp]
        L.dg_structure_function.argtypes = [vp, i, C.c_int64, C.c_uint64, vp, vp]
        L.dg_analysis_bytes.argtypes = [C.POINTER(Mesh), i, C.POINTER(C.c_size_t)]
        L.dg_power_spectrum.argtypes = [vp, vp, C.c_size_t, i, vp, vp, vp]
        _lib = L
    return _lib


# every symbol include/dg.h declares
EXPORTS = ("dg_scratch_bytes", "dg_vhat_bytes", "dg_init", "dg_free", "dg_last_error", "dg_set_state", "dg_get_state", "dg_rhs",
           "dg_project_velocity", "dg_step", "dg_set_forcing", "dg_set_forcing_coeffs", "dg_forcing_from_modes",
           "dg_diagnostics", "dg_l1_density", "dg_get_meta", "dg_set_meta", "dg_profile", "dg_profile_read",
           "dg_rhs_noalloc", "dg_av_param_count", "dg_set_av_weights", "dg_get_av_weights", "dg_generate_pairs",
           "dg_mlp_train", "dg_mlp_grad", "dg_mlp_forward", "dg_av_nu", "dg_av_nu_carried", "dg_density_pdf", "dg_structure_function",
           "dg_analysis_bytes", "dg_power_spectrum", "dg_adi_buffer_bytes", "dg_adi_init", "dg_adi_free",
           "dg_adi_last_error", "dg_adi_set_state", "dg_adi_get_state", "dg_adi_project", "dg_adi_rhs",
           "dg_adi_step", "dg_adi_totals", "dg_adi_set_forcing", "dg_adi_set_reset", "dg_adi_energy_budget",
           "dg_adi_get_meta", "dg_adi_set_meta")

MAX_BINS = 2000


class DGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (ERROR_NAMES.get(code, str(code)), msg))
        self.code = code
