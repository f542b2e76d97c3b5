"""The GPU discrete adjoint against the oracle's reverse mode, element by element.

The oracle tapes its own right-hand side (every elementary operation's adjoint written out,
pinned on the CPU by the transposed-tangent identity and by finite differences) and walks the
tape backwards; the CUDA adjoint is a hand-written reverse of the tiled sweeps.  On the same
seeded inputs their state and metric adjoints agree element by element: relative max-norm
max|gpu - oracle| / max|oracle| <= 1e-11.  Both are exact derivatives of the same operator in
FP64, evaluated in different orders; the adjoint of a right-hand side sums a few thousand
products per entry, so its rounding is a few hundred ulps of the largest contribution, and
the bar leaves an order of magnitude above what is measured.  Cases: a periodic grid whose
xi and eta tiles end ragged (140 x 40), every boundary kind, the smooth vortex with the
unmapped-weight epsilon, one RK3 step, and the metrics; WENOIU7-1MP (the Appendix's r = 4
interpolation) in each."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-11
GAMMA = 1.4


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


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _rhs_case(F, cfgd, x, y, q, seed):
    M = O.metrics(cfgd, x, y)
    g = np.random.default_rng(seed).standard_normal(q.shape)
    Qb_o, Mb_o = O.rhs_vjp(cfgd, M, q, g)
    Qb, Mb = F.rhs_vjp(F.Config.from_dict(cfgd), _dev(M), _dev(q), _dev(g))
    return _rel(_host(Qb), Qb_o), _rel(_host(Mb), Mb_o)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rhs_vjp_equals_oracle_ragged_tiles(F, scheme):
    x, y, per = I.periodic_square(140, 8.0, 0.2, seed=21, nj=40)
    q = I.random_state(x.shape, seed=31)
    eq, em = _rhs_case(F, dict(scheme=scheme, period=per), x, y, q, seed=scheme)
    assert eq <= TOL and em <= TOL, (eq, em)


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (3, 3, 3, 3), (2, 4, 3, 1), (4, 4, 4, 4)])
def test_rhs_vjp_equals_oracle_boundaries(F, bc):
    x, y = I.riemann_grid(24, 0.2, 4)
    q = I.random_state(x.shape, seed=32)
    st = np.array([I.conservative(1.0, 0.3, -0.2, 1.0 / GAMMA), I.conservative(0.9, -0.4, 0.1, 0.8),
                   I.conservative(1.1, 0.2, 0.5, 0.7), I.conservative(1.0, 0.0, -0.3, 0.75)])
    for scheme in (0, 2, 3, 4):
        eq, em = _rhs_case(F, dict(scheme=scheme, bc=bc, bc_state=st), x, y, q, seed=7)
        assert eq <= TOL and em <= TOL, (scheme, eq, em)


def test_rhs_vjp_equals_oracle_smooth_vortex(F):
    """The adjoint workload's setting: a smooth state with eps = 1e-6 (near-uniform far field)."""
    x, y, per = I.periodic_square(64, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    eq, em = _rhs_case(F, dict(scheme=2, period=per, eps=1e-6), x, y, q, seed=5)
    assert eq <= TOL and em <= TOL, (eq, em)


@pytest.mark.parametrize("scheme", [2, 4])
def test_rk3_step_vjp_equals_oracle(F, scheme):
    x, y, per = I.periodic_square(40, 8.0, 0.2, seed=21, nj=24)
    q = I.random_state(x.shape, seed=33)
    cfgd = dict(scheme=scheme, period=per)
    M = O.metrics(cfgd, x, y)
    g = np.random.default_rng(2).standard_normal(q.shape)
    dt = 0.02
    Qb_o, Mb_o = O.rk3_vjp(cfgd, M, q, dt, g)
    Qb, Mb = _dev(g), torch.zeros(M.shape, dtype=torch.float64, device="cuda")
    F.rk3_step_vjp(F.Config.from_dict(cfgd), _dev(M), _dev(q), dt, Qb, Mb)
    assert _rel(_host(Qb), Qb_o) <= TOL and _rel(_host(Mb), Mb_o) <= TOL


@pytest.mark.parametrize("scheme,bc", [(2, None), (0, (1, 1, 1, 1)), (3, (3, 2, 4, 1)), (4, None), (4, (1, 1, 1, 1))])
def test_metrics_vjp_equals_oracle(F, scheme, bc):
    if bc is None:
        x, y, per = I.periodic_square(36, 8.0, 0.2, seed=21, nj=28)
        cfgd = dict(scheme=scheme, period=per)
    else:
        x, y = I.riemann_grid(24, 0.2, 4)
        cfgd = dict(scheme=scheme, bc=bc)
    Mg = np.random.default_rng(3).standard_normal(O.metrics(cfgd, x, y).shape)
    xb_o, yb_o = O.metrics_vjp(cfgd, x, y, Mg)
    xb, yb = F.metrics_vjp(F.Config.from_dict(cfgd), _dev(x), _dev(y), _dev(Mg))
    assert _rel(_host(xb), xb_o) <= TOL and _rel(_host(yb), yb_o) <= TOL
