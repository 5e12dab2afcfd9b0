"""Positivity by repetition of the step on the GPU (Sec. 3.1, last paragraph),
through the C ABI, against the FP64 oracle.

The states are the driven start from rest (Mach-3 OU driving, seed 11) at the
step where the plain rescaling first troubles cells; their decisions (point
densities against the floor, wave speeds against 1.5 S) lie far from the
thresholds, so every precision marks the same cells.  Bounds as the plain
step parity: FP64 1e-12, FP32 3e-5, x3 1e-4 relative L2 per field.  The long
runs check that the repetition carries the driven start from rest past the
time where the rescaling alone breaks down (t ~ 0.1 at every resolution tried).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="no CUDA device")

from oracle import oracle as O  # noqa: E402
from paper_2401_06841_gb300 import Solver  # noqa: E402
from paper_2401_06841_gb300 import _lib as B  # noqa: E402

TOL = {"f64": 1e-12, "f32": 3e-5, "x3": 1e-4}


def rel_l2_fields(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return np.array([np.linalg.norm(got[:, v] - ref[:, v]) / max(np.linalg.norm(ref[:, v]), 1e-300)
                     for v in range(ref.shape[1])])


def driven_start(N, k, nsteps, seed=11):
    cfg = O.make_cfg(N, k)
    u = np.zeros((N ** 3, 4, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    rc, t, _, ah = O.run(cfg, u, nsteps, forcing=O.Forcing(mach=3.0, zeta=0.5, seed=seed))
    assert rc == 0
    return cfg, u, ah


@pytest.mark.gpu
@pytest.mark.parametrize("prec,k,n,backend", [("f64", 2, 40, "tcgen05"), ("f32", 2, 40, "tcgen05"),
                                              ("f64", 3, 51, "tcgen05"), ("x3", 3, 51, "tcgen05"),
                                              ("x3", 3, 51, "mma")])
def test_repeated_step_matches_the_oracle(prec, k, n, backend):
    N = 8
    cfg, u, ah = driven_start(N, k, n)
    ref = u.copy()
    st, dtu, att, lev = O.step_repeat(O.make_cfg(N, k, positivity="repeat"), ref, ah)
    assert st >= 0 and att >= 2 and lev.any()
    s = Solver(N, k, precision=prec, positivity="repeat", x3_backend=backend)
    s.set_state(u)
    s.set_forcing_coeffs(ah)
    _, dl = s.step(1)
    got = s.get_state().cpu().numpy()
    d = s.diagnostics()
    s.close()
    assert d["status"] & B.ST_REPEATED
    assert dl == pytest.approx(dtu, rel={"f64": 1e-13, "f32": 1e-6, "x3": 5e-5}[prec])
    err = rel_l2_fields(got, ref)
    assert err.max() < TOL[prec], err


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "x3"])
def test_untroubled_steps_are_the_plain_steps(prec):
    # a state whose steps trouble no cell: both modes give the same bits
    N, k = 8, 3
    _, u, ah = driven_start(N, k, 20)
    out = []
    for pos in ("scale", "repeat"):
        s = Solver(N, k, precision=prec, positivity=pos)
        s.set_state(u)
        s.set_forcing_coeffs(ah)
        s.step(3)
        out.append(s.get_state().cpu().numpy())
        assert not (s.diagnostics()["status"] & B.ST_REPEATED)
        s.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.gpu
@pytest.mark.timeout(600)
@pytest.mark.parametrize("N,k,prec", [(16, 2, "f32"), (16, 3, "x3"), (64, 3, "x3")])
def test_driven_start_from_rest_runs_through(N, k, prec):
    s = Solver(N, k, precision=prec, positivity="repeat")
    u = np.zeros((N ** 3, 4, O.nmodes(k)))
    u[:, 0, 0] = 1.0
    s.set_state(u)
    s.set_forcing(mach=3.0, zeta=0.5, seed=11)
    t, steps = 0.0, 0
    while t < 0.15:
        t, _ = s.step(10)
        steps += 10
        assert steps < 20000
    d = s.diagnostics()
    s.close()
    assert math.isfinite(d["max_speed"]) and d["max_speed"] < 100.0, d
    assert abs(d["mass"] - 1.0) < (1e-12 if prec == "f64" else 1e-4)
    assert d["status"] & B.ST_REPEATED
