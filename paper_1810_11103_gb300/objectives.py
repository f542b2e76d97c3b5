"""Scalar objectives for the adjoint of the shock-vortex case, written with torch
operations so that autograd supplies their partial derivatives (this is the user's
functional, not part of the scheme's arithmetic; it runs on CPU or GPU tensors).

J(Q, x, y, M) = sum_j p(0, j) ds_j                      pressure force on the outflow face i = 0
              + sum_{(i, j) in W} p(i, j) J^-1(i, j)     pressure integrated over a window of columns

ds_j is the trapezoid share of the boundary arc length at node j, from the node
coordinates, and J^-1 is the metric Jacobian (the cell area in computational units), so J
depends on the grid directly as well as through the flow.
"""
from __future__ import annotations

import numpy as np
import torch

G = 4          # ghost layers of the stored metrics


def pressure(Q: torch.Tensor, gamma: float = 1.4) -> torch.Tensor:
    return (gamma - 1.0) * (Q[3] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2]) / Q[0])


def window_of(x: np.ndarray, lo: float = -2.0, hi: float = 6.0):
    """Columns [i0, i1) whose first-row x lies in [lo, hi]."""
    xs = np.asarray(x)[0]
    idx = np.nonzero((xs >= lo) & (xs <= hi))[0]
    return int(idx[0]), int(idx[-1]) + 1


def terms(Q: torch.Tensor, x: torch.Tensor, y: torch.Tensor, M: torch.Tensor, window, gamma: float = 1.4):
    """The per-node contributions of J: (boundary terms (nj,), window terms (nj, i1 - i0))."""
    nj, ni = x.shape
    p = pressure(Q[:, :, :ni], gamma)
    dx = x[1:, 0] - x[:-1, 0]
    dy = y[1:, 0] - y[:-1, 0]
    half = 0.5 * torch.sqrt(dx * dx + dy * dy)
    z = half.new_zeros(1)
    ds = torch.cat([half, z]) + torch.cat([z, half])
    i0, i1 = window
    return p[:, 0] * ds, p[:, i0:i1] * M[4, G:G + nj, G + i0:G + i1]


def shock_vortex_functional(Q, x, y, M, window, gamma: float = 1.4) -> torch.Tensor:
    b, w = terms(Q, x, y, M, window, gamma)
    return b.sum() + w.sum()
