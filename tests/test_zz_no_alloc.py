"""dg_rhs_noalloc: the right-hand side for callers that cannot allocate device
memory (their memory is held by their own pool, or cudaMalloc/cudaFree would
synchronise a pipeline that must not stall).  Its working memory is a fixed
device array inside the library; these tests call it through the C ABI and
compare it with dg_rhs, which works on a context with caller-owned scratch.

The file name makes pytest collect it last; it also passes on its own in a
fresh process."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="no CUDA device")

from oracle import oracle as O  # noqa: E402
from paper_2401_06841_gb300 import Solver  # noqa: E402
from paper_2401_06841_gb300 import _lib as B  # noqa: E402
from paper_2401_06841_gb300 import inputs as I  # noqa: E402

PREC = {"f64": (B.PREC_F64, torch.float64, 1e-12), "f32": (B.PREC_F32, torch.float32, 1e-5),
        "x3": (B.PREC_X3, torch.float32, 5e-5)}


def rel_l2_fields(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.array([np.linalg.norm(got[:, v] - ref[:, v]) / max(np.linalg.norm(ref[:, v]), 1e-300)
                     for v in range(ref.shape[1])])


def noalloc_rhs(N, k, prec, u, ahat, dt, stream):
    L = B.lib()
    code, dtype, _ = PREC[prec]
    mesh = B.Mesh((C.c_int32 * 3)(N, N, N), (C.c_double * 3)(1.0, 1.0, 1.0))
    nu = B.NuParams(B.AV_VNR, 2.0, 0.2, 1e-3, 0.0)
    ud = torch.as_tensor(u, dtype=dtype).cuda().contiguous()
    ad = None if ahat is None else torch.as_tensor(ahat, dtype=dtype).cuda().contiguous()
    out = torch.full_like(ud, float("nan"))
    torch.cuda.synchronize()
    rc = L.dg_rhs_noalloc(C.byref(mesh), k, 1.0, C.byref(nu), code, ud.data_ptr(),
                          None if ad is None else ad.data_ptr(), out.data_ptr(), dt, stream.cuda_stream)
    assert rc == B.DG_OK
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_rhs_matches_dg_rhs_on_consecutive_calls():
    stream = torch.cuda.Stream()
    cases = [("f64", 5, 2, True), ("f32", 6, 3, False), ("x3", 6, 3, True), ("f64", 5, 2, False)]
    for i, (prec, N, k, forced) in enumerate(cases):
        u = I.random_state(N, k, seed=200 + i)
        a = None
        if forced:
            fo = O.Forcing(mach=2.0, zeta=0.5, seed=i)
            a = O.forcing_project(O.make_cfg(N, k), fo.kvec(), fo.amplitudes())
        dt = 0.3 * (1 / N) / ((k + 1) * 6.0)
        got = noalloc_rhs(N, k, prec, u, a, dt, stream)
        ref = Solver(N, k, precision=prec).rhs(u, a, dt).cpu().numpy()
        assert np.isfinite(got).all()
        err = rel_l2_fields(got, ref)
        assert err.max() <= PREC[prec][2], (prec, err)


@pytest.mark.gpu
def test_noalloc_rejects_meshes_beyond_the_fixed_array():
    L = B.lib()
    mesh = B.Mesh((C.c_int32 * 3)(128, 128, 128), (C.c_double * 3)(1.0, 1.0, 1.0))
    nu = B.NuParams(B.AV_VNR, 2.0, 0.2, 1e-3, 0.0)
    s = torch.cuda.Stream()
    # 128^3 cells x 60 floats of projected velocity = 503 MB > 64 MiB: refused
    # before any device work, so the buffers are never touched
    small = torch.zeros(16, device="cuda")
    rc = L.dg_rhs_noalloc(C.byref(mesh), 3, 1.0, C.byref(nu), B.PREC_F32, small.data_ptr(), None, small.data_ptr(),
                          0.0, s.cuda_stream)
    assert rc == B.DG_ENOMEM
