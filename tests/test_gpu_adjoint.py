"""Discrete adjoint on the GPU against the oracle's exact forward-mode tangent, by the
dot-product identity <gbar, J w> = <J^T gbar, w>: right-hand side (state and metric
adjoints, every boundary kind), metrics (coordinate adjoints), one RK3 step."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TOL = 1e-10


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _periodic_case(n=24, nj=20):
    x, y, per = I.periodic_square(n, 8.0, 0.2, seed=21, nj=nj)
    return x, y, per, I.random_state(x.shape, seed=31)


def _wall_case():
    x, y = I.riemann_grid(20, 0.2, 4)
    return x, y, ((0.0, 0.0), (0.0, 0.0)), I.random_state(x.shape, seed=32)


def _dot_check(F, cfgd, x, y, q, seed=0):
    rng = np.random.default_rng(seed)
    M = O.metrics(cfgd, x, y)
    g = rng.standard_normal(q.shape)
    dq = rng.standard_normal(q.shape)
    dM = rng.standard_normal(M.shape) * 0.01 * np.abs(M).max(axis=(1, 2), keepdims=True)
    _, dR = O.rhs_jvp(cfgd, M, q, dM, dq)
    cfg = F.Config.from_dict(cfgd)
    Qb, Mb = F.rhs_vjp(cfg, _dev(M), _dev(q), _dev(g))
    lhs = float((g * dR).sum())
    rhs = float((_host(Qb) * dq).sum() + (_host(Mb) * dM).sum())
    assert abs(lhs - rhs) < TOL * (abs(lhs) + np.abs(g).sum() * np.abs(dR).max() * 1e-6), (lhs, rhs)
    # the state part and the metric part separately
    _, dRq = O.rhs_jvp(cfgd, M, q, None, dq)
    assert abs(float((g * dRq).sum()) - float((_host(Qb) * dq).sum())) < TOL * abs(float((g * dRq).sum())) + 1e-12
    _, dRm = O.rhs_jvp(cfgd, M, q, dM, None)
    assert abs(float((g * dRm).sum()) - float((_host(Mb) * dM).sum())) < TOL * abs(float((g * dRm).sum())) + 1e-12


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rhs_vjp_periodic(F, scheme):
    x, y, per, q = _periodic_case()
    _dot_check(F, dict(scheme=scheme, period=per), x, y, q, seed=scheme)


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (3, 3, 3, 3), (2, 4, 3, 1), (4, 4, 4, 4)])
def test_rhs_vjp_boundaries(F, bc):
    x, y, per, q = _wall_case()
    st = np.tile(I.conservative(1.0, 0.3, -0.2, 1.0 / GAMMA), (4, 1))
    for scheme in (0, 3, 4):
        _dot_check(F, dict(scheme=scheme, bc=bc, bc_state=st), x, y, q, seed=7)


def test_rhs_vjp_options(F):
    x, y, per, q = _periodic_case(18, 16)
    for opt in (dict(interp=1), dict(linear_weights=1), dict(ppm=0, eps=1e-6)):
        _dot_check(F, dict(scheme=2, period=per, **opt), x, y, q, seed=3)


@pytest.mark.parametrize("scheme,bc", [(2, (0, 0, 0, 0)), (1, (1, 1, 3, 3)), (4, (1, 1, 3, 3))])
def test_metrics_vjp(F, scheme, bc):
    if bc[0] == 0:
        x, y, per = I.periodic_square(20, 8.0, 0.2, seed=5, nj=18)
    else:
        x, y = I.riemann_grid(20, 0.2, 6)
        per = ((0.0, 0.0), (0.0, 0.0))
    cfgd = dict(scheme=scheme, bc=bc, period=per)
    rng = np.random.default_rng(1)
    dx, dy = rng.standard_normal(x.shape), rng.standard_normal(y.shape)
    M, dM = O.metrics_jvp(cfgd, x, y, dx, dy)
    Mb = rng.standard_normal(M.shape)
    xb, yb = F.metrics_vjp(F.Config.from_dict(cfgd), _dev(x), _dev(y), _dev(Mb))
    lhs = float((Mb * dM).sum())
    rhs = float((_host(xb) * dx).sum() + (_host(yb) * dy).sum())
    assert abs(lhs - rhs) < 1e-11 * np.abs(Mb).sum() * np.abs(dM).max()


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_rk3_step_vjp(F, scheme):
    x, y, per, q = _periodic_case(20, 16)
    cfgd = dict(scheme=scheme, period=per)
    M = O.metrics(cfgd, x, y)
    rng = np.random.default_rng(2)
    dq = rng.standard_normal(q.shape)
    dM = rng.standard_normal(M.shape) * 0.01 * np.abs(M).max(axis=(1, 2), keepdims=True)
    dt = 0.3 * O.cfl_dt(cfgd, M, q, 1.0)
    _, dQ1 = O.rk3_jvp(cfgd, M, q, dq, dt, 1, dM)
    a = rng.standard_normal(q.shape)
    cfg = F.Config.from_dict(cfgd)
    Qb = _dev(a)
    Mb = torch.zeros_like(_dev(M))
    F.rk3_step_vjp(cfg, _dev(M), _dev(q), dt, Qb, Mb)
    lhs = float((a * dQ1).sum())
    rhs = float((_host(Qb) * dq).sum() + (_host(Mb) * dM).sum())
    assert abs(lhs - rhs) < TOL * (np.abs(a).sum() * np.abs(dQ1).max())


def test_recorded_step_matches_step_and_its_adjoint(F):
    x, y, per, q = _periodic_case(20, 16)
    cfgd = dict(scheme=3, period=per)
    cfg = F.Config.from_dict(cfgd)
    M = O.metrics(cfgd, x, y)
    dt = 0.3 * O.cfl_dt(cfgd, M, q, 1.0)
    Md, Q1, Q2 = _dev(M), _dev(q), _dev(q)
    F.rk3_step(cfg, Md, Q1, dt)
    tape = F.rk3_tape(cfg, Q2)
    F.rk3_step_record(cfg, Md, Q2, dt, tape)
    assert np.abs(_host(Q2) - _host(Q1)).max() < 1e-13 * np.abs(q).max()
    # the taped reverse equals the self-contained one
    a = np.random.default_rng(5).standard_normal(q.shape)
    Qa, Qb = _dev(a), _dev(a)
    Ma, Mb = torch.zeros_like(Md), torch.zeros_like(Md)
    F.rk3_step_vjp(cfg, Md, _dev(q), dt, Qa, Ma)
    F.rk3_step_vjp_tape(cfg, Md, tape, dt, Qb, Mb)
    assert np.abs(_host(Qa) - _host(Qb)).max() < 1e-12 * np.abs(_host(Qa)).max()
    assert np.abs(_host(Ma) - _host(Mb)).max() < 1e-12 * np.abs(_host(Ma)).max()
