"""Pins of the oracle's reverse mode (the Rev scalar's tape), CPU only.

The adjoint is the transpose of the tangent: for any seed g and direction w,
<g, J w> = <J^T g, w>, with J w from the oracle's dual-number tangent and J^T g from the tape.
Both are exact derivatives of the same floating-point computation, so they agree to rounding
wherever the computation is well conditioned: on states whose nodes are independent (every
smoothness indicator far above rounding) with eps = 1e-40, and on smooth states with the
unmapped-weight eps = 1e-6.  (Near exactly uniform data with eps = 1e-40 the weights are set
by rounding noise and their derivatives are O(1 / eps); there the two disagree at the 1e-3
level, which is why the adjoint workload takes eps = 1e-6.)  Finite differences pin the
adjoint independently of the tangent code."""
import numpy as np
import pytest

import oracle as O
from oracle import oracle as OO   # the functions (oracle.count_flops is also a submodule name)
from paper_1810_11103_gb300 import inputs as I

DOT_TOL = 1e-12


def _dot_rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def _grid(n=14, seed=21):
    return I.periodic_square(n, 8.0, 0.2, seed=seed)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("smooth", [False, True])
def test_rhs_vjp_is_the_transposed_tangent(scheme, smooth):
    # WENOIU7's 7-node stencils see the 14-node vortex as barely resolved, where the weights'
    # derivatives (b^-3 with eps = 1e-6) amplify rounding to 2e-11: its case takes 20 nodes
    x, y, per = _grid(20 if scheme == 4 else 14)
    if smooth:
        cfg = dict(scheme=scheme, period=per, eps=1e-6)
        q = I.isentropic_vortex(x, y, (4.0, 4.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(8.0, 8.0))
    else:
        cfg = dict(scheme=scheme, period=per)
        q = I.random_state(x.shape, seed=31)
    M = O.metrics(cfg, x, y)
    rng = np.random.default_rng(100 + scheme)
    g = rng.normal(size=q.shape)
    w = rng.normal(size=q.shape)
    wM = rng.normal(size=M.shape) * 0.05 * np.abs(M).max(axis=(1, 2), keepdims=True)
    Qb, Mb = O.rhs_vjp(cfg, M, q, g)
    _, dR = O.rhs_jvp(cfg, M, q, wM, w)
    assert _dot_rel(float((g * dR).sum()), float((Qb * w).sum() + (Mb * wM).sum())) < DOT_TOL
    # each part on its own
    _, dRq = O.rhs_jvp(cfg, M, q, None, w)
    assert _dot_rel(float((g * dRq).sum()), float((Qb * w).sum())) < DOT_TOL


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (3, 2, 4, 1)])
def test_rhs_vjp_with_boundaries(bc):
    x, y = I.riemann_grid(20, 0.3, 1811)
    q = I.random_state(x.shape, seed=5)
    st = np.array([[1.0, 0.3, -0.2, 2.6], [0.9, -0.1, 0.2, 2.4], [1.1, 0.5, 0.1, 2.8], [1.0, 0.0, 0.4, 2.5]])
    cfg = dict(scheme=2, bc=bc, bc_state=st)
    M = O.metrics(cfg, x, y)
    rng = np.random.default_rng(9)
    g, w = rng.normal(size=q.shape), rng.normal(size=q.shape)
    wM = rng.normal(size=M.shape) * 0.05 * np.abs(M).max(axis=(1, 2), keepdims=True)
    Qb, Mb = O.rhs_vjp(cfg, M, q, g)
    _, dR = O.rhs_jvp(cfg, M, q, wM, w)
    assert _dot_rel(float((g * dR).sum()), float((Qb * w).sum() + (Mb * wM).sum())) < DOT_TOL


def test_rk3_vjp_is_the_transposed_tangent():
    x, y, per = _grid(12)
    cfg = dict(scheme=2, period=per)
    q = I.random_state(x.shape, seed=31)
    M = O.metrics(cfg, x, y)
    rng = np.random.default_rng(4)
    g, w = rng.normal(size=q.shape), rng.normal(size=q.shape)
    wM = rng.normal(size=M.shape) * 0.05 * np.abs(M).max(axis=(1, 2), keepdims=True)
    Qb, Mb = O.rk3_vjp(cfg, M, q, 0.05, g)
    _, dQ1 = O.rk3_jvp(cfg, M, q, w, 0.05, 1, dM=wM)
    assert _dot_rel(float((g * dQ1).sum()), float((Qb * w).sum() + (Mb * wM).sum())) < DOT_TOL


@pytest.mark.parametrize("scheme", [0, 3, 4])
def test_metrics_vjp_is_the_transposed_tangent(scheme):
    x, y, per = _grid()
    cfg = dict(scheme=scheme, period=per)
    rng = np.random.default_rng(7)
    dx, dy = rng.normal(size=x.shape), rng.normal(size=y.shape)
    _, dM = O.metrics_jvp(cfg, x, y, dx, dy)
    Mg = rng.normal(size=dM.shape)
    xb, yb = O.metrics_vjp(cfg, x, y, Mg)
    assert _dot_rel(float((Mg * dM).sum()), float((xb * dx).sum() + (yb * dy).sum())) < DOT_TOL


def test_rhs_vjp_matches_finite_differences():
    """Independent of the tangent code: the gradient of <g, rhs> along random directions."""
    x, y, per = _grid()
    cfg = dict(scheme=2, period=per)
    q = I.random_state(x.shape, seed=31)
    M = O.metrics(cfg, x, y)
    rng = np.random.default_rng(11)
    g = rng.normal(size=q.shape)
    Qb, Mb = O.rhs_vjp(cfg, M, q, g)
    for k in range(3):
        w = rng.normal(size=q.shape)
        wM = rng.normal(size=M.shape) * 0.05 * np.abs(M).max(axis=(1, 2), keepdims=True)
        e = 1e-6
        fd = ((g * (O.rhs(cfg, M + e * wM, q + e * w) - O.rhs(cfg, M - e * wM, q - e * w))).sum()) / (2 * e)
        assert _dot_rel(float(fd), float((Qb * w).sum() + (Mb * wM).sum())) < 1e-6


def test_vjp_operation_count():
    """The reverse sweep's count: every tape record except the leaves has one or two operand
    edges of one or two operations each; the forward part is the right-hand side's own count."""
    x, y, per = _grid(12)
    cfg = dict(scheme=2, period=per)
    q = I.random_state(x.shape, seed=3)
    M = O.metrics(cfg, x, y)
    c = O.count_vjp_flops(cfg, M, q)
    ops = c["records"] - (M.size + q.size)
    assert 0 < ops <= c["reverse"] <= 4 * ops
    assert c["forward"] == OO.count_flops(cfg, M, q)
    assert 0 < c["partials"] < c["forward"]


def test_vjp_count_affine_in_line_length():
    """With the line count fixed, the count is affine in the line length (each line is the same
    program); with linear weights no data-dependent branch (the mapping's two sides) changes it,
    so the affinity is exact.  This lets the stored per-node figure be evaluated at the
    workload's size from two smaller grids."""
    tot = []
    for ni in (16, 24, 32):
        x, y, per = I.periodic_square(ni, 8.0, 0.2, seed=21, nj=12)
        q = I.random_state(x.shape, seed=3)
        cfg = dict(scheme=2, period=per, linear_weights=1)
        c = O.count_vjp_flops(cfg, O.metrics(cfg, x, y), q)
        tot.append(c["forward"] + c["partials"] + c["reverse"])
    assert tot[2] - tot[1] == tot[1] - tot[0] > 0
