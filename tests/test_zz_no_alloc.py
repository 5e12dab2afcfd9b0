"""dg_rhs_noalloc: the right-hand side for callers that cannot allocate device
memory (their memory is held by their own pool, or cudaMalloc/cudaFree would
synchronise a pipeline that must not stall).  Its working memory is a fixed
device array inside the library.  These tests call it through the C ABI and
compare it with the FP64 oracle on the same inputs (whole mesh on small
meshes, sampled cells at the largest mesh the array holds), on consecutive
calls, and bit for bit with dg_rhs on a context running the same kernel; both
sides of the size limit are checked.

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
def test_noalloc_rhs_matches_the_oracle_on_consecutive_calls():
    stream = torch.cuda.Stream()
    cases = [("f64", 5, 2, True), ("f32", 6, 3, False), ("x3", 6, 3, True), ("f64", 5, 2, False), ("x3", 7, 1, True)]
    for i, (prec, N, k, forced) in enumerate(cases):
        u = I.random_state(N, k, seed=200 + i)
        cfg = O.make_cfg(N, k)
        a = None
        if forced:
            fo = O.Forcing(mach=2.0, zeta=0.5, seed=i)
            a = O.forcing_project(cfg, fo.kvec(), fo.amplitudes())
        dt = 0.3 * (1 / N) / ((k + 1) * 6.0)
        ref = O.rhs(cfg, u, a, dt)
        for call in range(2):
            got = noalloc_rhs(N, k, prec, u, a, dt, stream)
            assert np.isfinite(got).all()
            err = rel_l2_fields(got, ref)
            assert err.max() <= PREC[prec][2], (prec, call, err)
        # and the context path on the same inputs: the same tile kernel, the same
        # tables (one builder for both paths), ordered reductions -- the same bits
        ctx = Solver(N, k, precision=prec, x3_backend="mma").rhs(u, a, dt).cpu().numpy()
        assert np.array_equal(got, ctx), (prec, N, k, np.abs(got - ctx).max())


# the array holds N^3 * 3 * b * element size bytes of projected velocity after a
# fixed 1,180,160-byte head (control block, reduction partials, tables)
LIMIT, HEAD = 64 << 20, 1180160


@pytest.mark.gpu
def test_noalloc_at_the_largest_mesh_it_holds():
    # k = 3 in FP32: N = 65 fits (66.0 MB + head <= 64 MiB), N = 66 does not
    N, k = 65, 3
    assert N ** 3 * 3 * 20 * 4 + HEAD <= LIMIT < (N + 1) ** 3 * 3 * 20 * 4 + HEAD
    stream = torch.cuda.Stream()
    u = I.random_state(N, k, seed=7)
    cfg = O.make_cfg(N, k)
    fo = O.Forcing(mach=2.0, zeta=0.5, seed=3)
    a = O.forcing_project(cfg, fo.kvec(), fo.amplitudes())
    dt = 0.3 * (1 / N) / ((k + 1) * 6.0)
    got = noalloc_rhs(N, k, "f32", u, a, dt, stream)
    assert np.isfinite(got).all()
    # sampled cells against the oracle (including the first and last cells and a
    # periodic corner), with the whole field's mean acceleration
    rng = np.random.default_rng(0)
    cells = np.unique(np.concatenate([[0, N - 1, N * N * N - 1, N * N * (N - 1)],
                                      rng.integers(0, N ** 3, 300)]))
    abar = O.forcing_mean(cfg, u, a)
    ref = O.rhs_cells(cfg, u, cells, a, abar, dt)
    assert rel_l2_fields(got[cells], ref).max() <= PREC["f32"][2]


@pytest.mark.gpu
def test_noalloc_rejects_meshes_beyond_the_fixed_array():
    L = B.lib()
    nu = B.NuParams(B.AV_VNR, 2.0, 0.2, 1e-3, 0.0)
    s = torch.cuda.Stream()
    small = torch.zeros(16, device="cuda")
    # refused before any device work, so the (too small) buffers are never touched
    for N, k, prec in [(66, 3, B.PREC_F32), (128, 3, B.PREC_F32), (52, 3, B.PREC_F64)]:
        assert N ** 3 * 3 * 20 * (8 if prec == B.PREC_F64 else 4) + HEAD > LIMIT
        mesh = B.Mesh((C.c_int32 * 3)(N, N, N), (C.c_double * 3)(1.0, 1.0, 1.0))
        rc = L.dg_rhs_noalloc(C.byref(mesh), k, 1.0, C.byref(nu), prec, small.data_ptr(), None,
                              small.data_ptr(), 0.0, s.cuda_stream)
        assert rc == B.DG_ENOMEM, (N, k, prec)
