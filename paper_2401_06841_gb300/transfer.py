"""Exact transfer of modal DG states between an N^3 mesh and its 2N^3
refinement, for accuracy comparisons (evaluation utility, not on the
solver's path).

A coarse cell holds 8 children; child s = (sx, sy, sz) occupies the half
[-1,0] (s=0) or [0,1] (s=1) of each coarse reference axis, so a coarse
coordinate is xi_c = (xi_f + 2s - 1)/2.  With the 1D matrices
    A[s][i][j] = (1/2) int_{-1}^{1} Pn_j(t) Pn_i((t + 2s - 1)/2) dt
(coarse degree i, fine degree j; exact Gauss-Legendre quadrature), the
child's coefficients of a coarse polynomial are f_m = sum_l c_l T[l][m] with
T = prod_d A[s_d][i_d(l)][j_d(m)] (exact: a degree-k polynomial stays degree
k under the affine map), and the L2 projection of a fine field back onto the
coarse cell is c_l = (1/8) sum_children sum_m T[l][m] f_m.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .inputs import mode_degrees


def _pn(m: int, x: np.ndarray) -> np.ndarray:
    c = np.zeros(m + 1)
    c[m] = 1.0
    return math.sqrt(2 * m + 1) * np.polynomial.legendre.legval(x, c)


def child_matrices(k: int) -> np.ndarray:
    """T[child][l][m] for the 8 children (child = sx + 2 sy + 4 sz)."""
    t, w = np.polynomial.legendre.leggauss(k + 2)
    A = np.zeros((2, k + 1, k + 1))
    for s in range(2):
        xc = (t + 2 * s - 1) / 2
        for i in range(k + 1):
            for j in range(k + 1):
                A[s, i, j] = 0.5 * np.sum(w * _pn(j, t) * _pn(i, xc))
    ijl = mode_degrees(k)
    b = len(ijl)
    T = np.zeros((8, b, b))
    for ch in range(8):
        s = (ch & 1, (ch >> 1) & 1, (ch >> 2) & 1)
        for l in range(b):
            for m in range(b):
                T[ch, l, m] = (A[s[0], ijl[l, 0], ijl[m, 0]] * A[s[1], ijl[l, 1], ijl[m, 1]]
                               * A[s[2], ijl[l, 2], ijl[m, 2]])
    return T


def _child_index(N: int, device):
    """fine cell index [coarse cell][child] on the 2N mesh."""
    iz, iy, ix = torch.meshgrid(torch.arange(N, device=device), torch.arange(N, device=device),
                                torch.arange(N, device=device), indexing="ij")
    ix, iy, iz = ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)
    out = []
    M = 2 * N
    for ch in range(8):
        sx, sy, sz = ch & 1, (ch >> 1) & 1, (ch >> 2) & 1
        out.append(((2 * iz + sz) * M + (2 * iy + sy)) * M + (2 * ix + sx))
    return torch.stack(out, dim=1)


def prolong(u: torch.Tensor, N: int, k: int) -> torch.Tensor:
    """N^3 state [N^3][4][b] -> exact 2N^3 state."""
    T = torch.as_tensor(child_matrices(k), dtype=u.dtype, device=u.device)
    idx = _child_index(N, u.device)
    fine = torch.empty((8 * N ** 3,) + tuple(u.shape[1:]), dtype=u.dtype, device=u.device)
    for ch in range(8):
        fine[idx[:, ch]] = torch.einsum("cvl,lm->cvm", u, T[ch])
    return fine


def restrict(uf: torch.Tensor, N: int, k: int) -> torch.Tensor:
    """2N^3 state -> L2 projection on the N^3 mesh."""
    T = torch.as_tensor(child_matrices(k), dtype=uf.dtype, device=uf.device)
    idx = _child_index(N, uf.device)
    out = torch.zeros((N ** 3,) + tuple(uf.shape[1:]), dtype=uf.dtype, device=uf.device)
    for ch in range(8):
        out += torch.einsum("cvm,lm->cvl", uf[idx[:, ch]], T[ch])
    return out / 8.0
