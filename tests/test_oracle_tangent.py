"""Pins of the oracle's forward-mode tangents (used to check the CUDA adjoint) against
central finite differences of the oracle itself (CPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I


def _case(scheme, n=14):
    x, y, per = I.periodic_square(n, 8.0, 0.2, seed=21)
    cfg = dict(scheme=scheme, period=per)
    # every node independent: the smoothness indicators stay far above the finite-difference
    # step everywhere, so the nonlinear weights are differentiable at the scale probed
    q = I.random_state(x.shape, seed=31)
    return cfg, x, y, q


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_rhs_tangent_matches_finite_differences(scheme):
    cfg, x, y, q = _case(scheme)
    M = O.metrics(cfg, x, y)
    rng = np.random.default_rng(scheme)
    dq = rng.normal(size=q.shape) * np.array([1.0, 1.0, 1.0, 2.0])[:, None, None]
    dM = rng.normal(size=M.shape) * 0.05 * np.abs(M).max(axis=(1, 2), keepdims=True)
    dM[4] = 0.0 * dM[4] + 0.01 * np.abs(M[4]).max() * rng.normal(size=M[4].shape)
    R, dR = O.rhs_jvp(cfg, M, q, dM, dq)
    assert np.array_equal(R, O.rhs(cfg, M, q))
    e = 1e-6
    fd = (O.rhs(cfg, M + e * dM, q + e * dq) - O.rhs(cfg, M - e * dM, q - e * dq)) / (2 * e)
    assert _rel(dR, fd) < 1e-6


@pytest.mark.parametrize("scheme", [0, 3])
def test_metrics_tangent_matches_finite_differences(scheme):
    cfg, x, y, _ = _case(scheme)
    rng = np.random.default_rng(7)
    dx, dy = rng.normal(size=x.shape), rng.normal(size=y.shape)
    M, dM = O.metrics_jvp(cfg, x, y, dx, dy)
    e = 1e-6
    fd = (O.metrics(cfg, x + e * dx, y + e * dy) - O.metrics(cfg, x - e * dx, y - e * dy)) / (2 * e)
    assert np.allclose(M, O.metrics(cfg, x, y), rtol=0, atol=0)
    assert _rel(dM, fd) < 1e-7


def test_rk3_tangent_matches_finite_differences():
    cfg, x, y, q = _case(2, n=12)
    M = O.metrics(cfg, x, y)
    rng = np.random.default_rng(3)
    dq = rng.normal(size=q.shape)
    Q1, dQ1 = O.rk3_jvp(cfg, M, q, dq, 0.05, 3)
    e = 1e-6
    fd = (O.rk3(cfg, M, q + e * dq, 0.05, 3) - O.rk3(cfg, M, q - e * dq, 0.05, 3)) / (2 * e)
    assert np.array_equal(Q1, O.rk3(cfg, M, q, 0.05, 3))
    assert _rel(dQ1, fd) < 1e-6
