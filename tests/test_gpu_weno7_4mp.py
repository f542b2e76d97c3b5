"""WENOIU7-4MP (the Appendix's scheme (3), four midpoints) on the GPU against the oracle.

The scheme's midpoint fluxes reach six nodes beyond a face, so it is built for periodic
blocks (ghost metrics beyond the stored four layers wrap) through the single-block entry
points, in FP64 and FP32.  Bars as for the other schemes: FP64 relative max-norm <= 1e-12
for metrics, right-hand sides and RK3 states; FP32 <= 1e-4 against the FP64 oracle on the
float-rounded state.  Every other use is refused."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

S74 = 5
TOL = 1e-12
GAMMA = 1.4


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("shape,smooth", [((256, 256), True), ((300, 70), True), ((97, 41), False)])
def test_metrics_and_rhs_parity(F, shape, smooth):
    ni, nj = shape
    x, y, per = I.periodic_square(ni, 10.0, 0.2, seed=1810, nj=nj)
    q = (I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
         if smooth else I.random_state(x.shape, seed=4))
    cfgd = dict(scheme=S74, period=per)
    cfg = F.Config.from_dict(cfgd)
    M_o = O.metrics(cfgd, x, y)
    M_g = _host(F.metrics(cfg, _dev(x), _dev(y)))
    assert np.abs(M_g[:4] - M_o[:4]).max() < TOL * np.abs(M_o[:4]).max()
    assert np.abs(M_g[4] - M_o[4]).max() < TOL * np.abs(M_o[4]).max()
    R_o = O.rhs(cfgd, M_o, q)
    assert _rel(_host(F.rhs(cfg, _dev(M_o), _dev(q))), R_o) < TOL


def test_rk3_and_free_stream(F):
    x, y, per = I.periodic_square(64, 8.0, 0.2, seed=21, nj=40)
    q = I.random_state(x.shape, seed=33)
    cfgd = dict(scheme=S74, period=per)
    cfg = F.Config.from_dict(cfgd)
    M = O.metrics(cfgd, x, y)
    q_o = O.rk3(cfgd, M, q, 0.01, 2)
    Q = _dev(q)
    for _ in range(2):
        F.rk3_step(cfg, _dev(M), Q, 0.01)
    assert _rel(_host(Q), q_o) < TOL
    Mg = F.metrics(cfg, _dev(x), _dev(y))
    q0 = _dev(I.uniform_state(x.shape, 1.0, 0.5, 0.3, 1.0 / GAMMA))
    assert float(F.rhs(cfg, Mg, q0).abs().max()) < 1e-12


def test_options(F):
    """WENO-Z weights and the midpoint splittings act on the interfaces only."""
    x, y, per = I.periodic_square(97, 12.0, 0.2, seed=8, nj=41)
    q = I.isentropic_vortex(x, y, (6.0, 6.0), strength=4.0, free=(1.0, 0.7, -0.4, 1.0), period=(12.0, 12.0))
    for opt in (dict(weights=1), dict(mid_split=2), dict(linear_weights=1), dict(interp=1)):
        cfgd = dict(scheme=S74, period=per, **opt)
        M = O.metrics(cfgd, x, y)
        assert _rel(_host(F.rhs(F.Config.from_dict(cfgd), _dev(M), _dev(q))), O.rhs(cfgd, M, q)) < TOL, opt


def test_fp32(F):
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    q32 = q.astype(np.float32).astype(np.float64)
    cfgd = dict(scheme=S74, period=per)
    M = O.metrics(cfgd, x, y)
    Rg = F.rhs(F.Config.from_dict(dict(cfgd, precision=1)), _dev(M), _dev(q32, torch.float32))
    assert Rg.dtype == torch.float32
    assert _rel(_host(Rg), O.rhs(cfgd, M, q32)) < 1e-4


def test_refusals(F):
    x, y, per = I.periodic_square(40, 8.0, 0.2, seed=21, nj=24)
    q = I.random_state(x.shape, seed=3)
    M, Q = _dev(O.metrics(dict(scheme=2, period=per), x, y)), _dev(q)
    for cfgd, code in ((dict(scheme=S74, bc=(1, 1, 0, 0)), 2), (dict(scheme=S74, period=per, precision=2), 2),
                       (dict(scheme=S74, period=per, scheme_alpha=1.2), 1)):
        with pytest.raises(F.FspError) as e:
            F.rhs(F.Config.from_dict(cfgd), M, Q.float() if cfgd.get("precision") else Q)
        assert e.value.code == code, cfgd
    with pytest.raises(F.FspError) as e:
        F.rhs_vjp(F.Config.from_dict(dict(scheme=S74, period=per)), M, Q, torch.ones_like(Q))
    assert e.value.code == 2
    with pytest.raises(F.FspError) as e:
        F.Batch(F.Config.from_dict(dict(scheme=S74)), [dict(x=x, y=y, bc=(0, 0, 0, 0), period=per)], [q])
    assert e.value.code == 2
