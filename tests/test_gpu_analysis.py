"""Parity of the GPU turbulence statistics (density PDF, structure function,
power spectrum; Sec. 4.1 and 4.3) with the oracle, through the C ABI, on the
same seeded states.  Both sides evaluate in FP64 from the same coefficients
(FP32 states are handed to the oracle as their FP32 values), so bin
decisions agree; sums differ only in their order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = pytest.mark.skip(reason="no CUDA device")

from oracle import oracle as O  # noqa: E402
from paper_2401_06841_gb300 import Solver  # noqa: E402
from paper_2401_06841_gb300 import inputs as I  # noqa: E402


def state(N, k, seed, prec):
    u = I.random_state(N, k, seed=seed, v_rms=0.8)
    if prec == "f32":
        u = u.astype(np.float32).astype(np.float64)
    return u


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_density_pdf_parity(k, prec):
    N = 5
    u = state(N, k, 70 + k, prec)
    s = Solver(N, k, precision=prec)
    s.set_state(u)
    got = s.density_pdf(-1.0, 1.0, 120)
    ref = O.density_pdf(O.make_cfg(N, k), u, -1.0, 1.0, 120)
    assert abs(ref.sum() - 1.0) < 1e-6
    assert np.abs(got - ref).max() < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3])
def test_structure_function_parity(k, prec):
    N = 6
    u = state(N, k, 80 + k, prec)
    s = Solver(N, k, precision=prec)
    s.set_state(u)
    l, v = s.structure_function(nbins=9, npairs=700, seed=123)
    lr, vr = O.structure_function(O.make_cfg(N, k), u, 9, 700, 123)
    assert np.allclose(l, lr, rtol=1e-14, atol=0)
    assert np.allclose(v, vr, rtol=1e-11, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("N,k", [(8, 3), (5, 2), (7, 1)])
def test_power_spectrum_parity(N, k):
    # Ng = 32 (even, with a Nyquist plane), 15 and 14
    u = state(N, k, 90 + k, "f64")
    s = Solver(N, k, precision="f64")
    s.set_state(u)
    km, pw, cnt = s.power_spectrum(60)
    kr, pr, cr = O.power_spectrum(O.make_cfg(N, k), u, 60)
    assert np.array_equal(cnt, cr)
    assert np.allclose(km, kr, rtol=1e-13, atol=0)
    assert np.allclose(pw, pr, rtol=1e-10, atol=1e-18 * pr.max())


@pytest.mark.gpu
def test_power_spectrum_single_mode_at_size():
    # v_y = A sin(2 pi x) on 32^3 cells at k = 3 (Ng = 128): the power A^2/2
    # sits in the first shell; FP32 state
    N, k, A = 32, 3, 0.4
    b = I.nmodes(k)
    u = np.zeros((N ** 3, 4, b))
    u[:, 0, 0] = 1.0
    u[:, 2, :] = A * I.fourier_coeffs(N, k, (1, 0, 0)).imag
    s = Solver(N, k, precision="f32")
    s.set_state(u)
    km, pw, cnt = s.power_spectrum(200)
    Ng = (k + 1) * N
    assert cnt.sum() == Ng ** 3 - 1 and cnt[0] == 6
    assert abs(pw[0] / (A * A / 2) - 1) < 1e-5
    assert pw[1:].sum() < 1e-6 * pw[0]
    # structure function of the same field: (1/2) A^2 (1 - sin(2 pi l)/(2 pi l)) in expectation
    l, v = s.structure_function(nbins=10, npairs=20000, seed=3)
    ref = np.sqrt(0.5 * A * A * (1 - np.sin(2 * np.pi * l) / (2 * np.pi * l)))
    assert np.all(np.abs(v / ref - 1) < 0.03), v / ref
    # uniform density: the PDF is a single bin
    h = s.density_pdf(-0.5, 0.5, 100)
    assert abs(h[50] - 1.0) < 1e-12
