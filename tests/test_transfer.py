"""Mesh transfer used by the accuracy comparison: prolongation is exact for
the coarse polynomial (checked pointwise with numpy's Legendre series) and
restriction inverts it; restriction of a fine field matches its Gauss L2
projection on the coarse cells."""
import math

import numpy as np
import torch

from paper_2401_06841_gb300 import inputs as I
from paper_2401_06841_gb300 import transfer as Tr


def _eval(coef, k, xi):
    ijl = I.mode_degrees(k)
    out = 0.0
    for l, (i, j, m) in enumerate(ijl):
        p = 1.0
        for deg, x in zip((i, j, m), xi):
            c = np.zeros(deg + 1)
            c[deg] = 1
            p *= math.sqrt(2 * deg + 1) * np.polynomial.legendre.legval(x, c)
        out += coef[l] * p
    return out


def test_prolongation_is_exact_and_restriction_inverts_it():
    N, k = 2, 3
    u = torch.as_tensor(I.random_state(N, k, seed=3))
    uf = Tr.prolong(u, N, k)
    rng = np.random.default_rng(0)
    for _ in range(20):
        X = rng.uniform(0, 1, 3)
        ic = np.floor(X * N).astype(int)
        xc = 2 * (X * N - ic) - 1
        iF = np.floor(X * 2 * N).astype(int)
        xf = 2 * (X * 2 * N - iF) - 1
        c = (ic[2] * N + ic[1]) * N + ic[0]
        f = (iF[2] * 2 * N + iF[1]) * 2 * N + iF[0]
        for v in range(4):
            assert abs(_eval(u[c, v].numpy(), k, xc) - _eval(uf[f, v].numpy(), k, xf)) < 1e-12
    back = Tr.restrict(uf, N, k)
    assert torch.allclose(back, u, atol=1e-13, rtol=0)


def test_restriction_of_a_fine_field_is_its_l2_projection():
    # the mean of each coarse cell equals the mean of its 8 children
    N, k = 2, 2
    uf = torch.as_tensor(I.random_state(2 * N, k, seed=4))
    uc = Tr.restrict(uf, N, k)
    idx = Tr._child_index(N, "cpu")
    assert torch.allclose(uc[:, :, 0], uf[idx][:, :, :, 0].mean(dim=1), atol=1e-14, rtol=0)
