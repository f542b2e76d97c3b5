"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element on
the same seeded inputs.  FP64 bar: relative max-norm max|gpu - oracle| / max|oracle|
<= 1e-12 for right-hand sides and RK3 states; for metrics the same bar, the four metric
planes against their common maximum and J^-1 against its own.  The
metrics are differences of O(1) coordinates that come out O(h), so their rounding is
O(eps / h) relative: about 4e-13 at h = 1/1023 with both sides correctly rounded."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-12
TOL_MET = 1e-12
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


def _cfg(**kw):
    c = dict(scheme=2, interp=0, ppm=1, linear_weights=0, bc=(0, 0, 0, 0), gamma=GAMMA, lf_alpha=1.1,
             eps=1e-40, period=((0.0, 0.0), (0.0, 0.0)), bc_state=None)
    c.update(kw)
    return c


def _vortex256():
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    return x, y, per, q


def _ragged(ni=300, nj=70, seed=5):
    # a 12 x 12 periodic box with ni x nj nodes: tiles of the sweeps end ragged
    x, y, per = I.periodic_square(ni, 12.0, 0.2, seed=seed, nj=nj)
    q = I.isentropic_vortex(x, y, (6.0, 6.0), strength=4.0, free=(1.0, 0.7, -0.4, 1.0), period=(12.0, 12.0))
    return x, y, per, q


def _riemann(n=60, seed=1811):
    x, y = I.riemann_grid(n, 0.3, seed)
    q = I.riemann_quadrants(x, y)
    return x, y, ((0.0, 0.0), (0.0, 0.0)), q


def _check_case(F, cfgd, x, y, q, tol=TOL_RHS):
    cfg = F.Config.from_dict(cfgd)
    M_o = O.metrics(cfgd, x, y)
    M_g = F.metrics(cfg, _dev(x), _dev(y))
    Mh = _host(M_g)
    # the four metric planes are coordinate derivatives of one scale; J^-1 has its own.
    # Every intermediate of a metric is a combination of coordinates, so each side rounds at
    # a few ulps of the largest coordinate X (the coefficients' absolute sum is about 3):
    # an absolute floor of 32 eps X on the planes, and through the two products of J^-1
    # 4 x that floor x the largest metric.  It matters only for lines far from the origin.
    X = max(np.abs(x).max(), np.abs(y).max())
    floor = 32 * np.finfo(np.float64).eps * X
    m4 = np.abs(M_o[:4]).max()
    assert np.abs(Mh[:4] - M_o[:4]).max() < TOL_MET * m4 + floor
    assert np.abs(Mh[4] - M_o[4]).max() < TOL_MET * np.abs(M_o[4]).max() + 4 * floor * m4
    R_o = O.rhs(cfgd, M_o, q)
    R_g = F.rhs(cfg, _dev(M_o), _dev(q))
    err = _rel(_host(R_g), R_o)
    assert err < tol, err
    return err


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rhs_parity_vortex_256(F, scheme):
    x, y, per, q = _vortex256()
    _check_case(F, _cfg(scheme=scheme, period=per), x, y, q)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rhs_parity_ragged_tiles(F, scheme):
    x, y, per, q = _ragged()
    _check_case(F, _cfg(scheme=scheme, period=per), x, y, q)


@pytest.mark.parametrize("variant", [dict(interp=1), dict(linear_weights=1), dict(ppm=0, eps=1e-6),
                                     dict(lf_alpha=1.2)])
def test_rhs_parity_options(F, variant):
    x, y, per, q = _ragged(97, 41, seed=8)
    for scheme in (0, 3):
        _check_case(F, _cfg(scheme=scheme, period=per, **variant), x, y, q)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rhs_parity_transmissive_riemann(F, scheme):
    x, y, per, q = _riemann()
    _check_case(F, _cfg(scheme=scheme, bc=(1, 1, 1, 1)), x, y, q)


def test_rhs_parity_boundary_kinds(F):
    x, y, per, q = _riemann(48, seed=3)
    # a different state on every face, so that each face must read its own (the far-field
    # velocities enter through some faces and leave through others)
    st = np.stack([I.conservative(1.0, 0.8, 0.3, 1.0 / GAMMA), I.conservative(1.1, 0.7, 0.2, 0.8),
                   I.conservative(0.9, -0.5, 0.1, 0.75), I.conservative(1.05, 0.6, -0.3, 0.7)])
    for bc in [(2, 2, 3, 3), (4, 4, 4, 4), (3, 4, 2, 1), (1, 3, 4, 2), (2, 2, 2, 2)]:
        for scheme in (1, 2):
            _check_case(F, _cfg(scheme=scheme, bc=bc, bc_state=st), x, y, q)
    # periodic in one direction, walls in the other
    xs, ys, per, qs = _ragged(64, 30, seed=2)
    _check_case(F, _cfg(scheme=3, bc=(0, 0, 3, 3), period=((12.0, 0.0), (0.0, 0.0))), xs, ys, qs)


def test_rhs_parity_one_dimensional(F):
    x, y, q, per = I.sod_1d(200)
    for scheme in range(4):
        _check_case(F, _cfg(scheme=scheme, bc=(1, 1, 0, 0), period=per), x, y, q)


def test_rhs_parity_smallest_blocks(F):
    # a single node per line in one direction, and the smallest non-periodic extent
    x, y, per = I.periodic_square(1, 1.0, 0.0, seed=0, nj=7)
    per = ((1.0, 0.0), (0.0, 1.0))
    q = I.random_state(x.shape, seed=4)
    _check_case(F, _cfg(scheme=3, period=per), x, y, q)
    xr, yr = I.riemann_grid(9, 0.2, 7)
    _check_case(F, _cfg(scheme=2, bc=(1, 1, 1, 1)), xr, yr, I.riemann_quadrants(xr, yr))


def test_line_lambda_and_cfl_parity(F):
    x, y, per, q = _ragged()
    cfgd = _cfg(scheme=2, period=per)
    cfg = F.Config.from_dict(cfgd)
    M = O.metrics(cfgd, x, y)
    lx_o, le_o = O.line_lambda(cfgd, M, q)
    lx_g, le_g = F.line_lambda(cfg, _dev(M), _dev(q))
    # the kernels return the maxima; the oracle includes the factor lf_alpha
    assert _rel(1.1 * _host(lx_g), lx_o) < 1e-14
    assert _rel(1.1 * _host(le_g), le_o) < 1e-14
    dt_g = float(_host(F.cfl_dt(cfg, _dev(M), _dev(q), 0.5))[0])
    assert dt_g == pytest.approx(O.cfl_dt(cfgd, M, q, 0.5), rel=1e-14)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rk3_parity(F, scheme):
    x, y, per, q = _ragged(96, 40, seed=6)
    cfgd = _cfg(scheme=scheme, period=per)
    cfg = F.Config.from_dict(cfgd)
    M = O.metrics(cfgd, x, y)
    dt = 0.5 * O.cfl_dt(cfgd, M, q, 1.0)
    q_o = O.rk3(cfgd, M, q, dt, 3)
    Qg = _dev(q)
    Mg = _dev(M)
    ws = F.workspace(cfg, Qg)
    for _ in range(3):
        F.rk3_step(cfg, Mg, Qg, dt, ws=ws)
    assert _rel(_host(Qg) - q, q_o - q) < 1e-11   # compare the change over the steps
    assert _rel(_host(Qg), q_o) < TOL_RHS


def test_free_stream_residual_on_gpu(F):
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q0 = np.array([1.0, 1.0, 1.0, 1.0 / (GAMMA - 1) + 1.0])
    for scheme in range(5):
        cfgd = _cfg(scheme=scheme, period=per)
        cfg = F.Config.from_dict(cfgd)
        Mg = F.metrics(cfg, _dev(x), _dev(y))
        R = _host(F.rhs(cfg, Mg, _dev(I.uniform_state(x.shape, 1.0, 1.0, 1.0, 1.0))))
        r_o = O.fsp_residual(cfgd, x, y, q0)
        assert np.abs(R).max() < 4 * r_o + 1e-14


def test_norms(F):
    rng = np.random.default_rng(0)
    a = rng.normal(size=(4, 33, 45))
    b = rng.normal(size=(4, 33, 45))
    out = _host(F.norms(_dev(a), _dev(b)))
    e = a - b
    for v in range(4):
        assert out[2 * v] == pytest.approx(math.sqrt((e[v] ** 2).mean()), rel=1e-12)
        assert out[2 * v + 1] == pytest.approx(np.abs(e[v]).max(), rel=0)


def test_argument_errors(F):
    x, y, per, q = _ragged(40, 20)
    cfg = F.Config.from_dict(_cfg(period=per))
    Qg = _dev(q)
    Mg = F.metrics(cfg, _dev(x), _dev(y))
    with pytest.raises(F.FspError) as e:       # host memory is refused
        F.rhs(cfg, Mg, torch.as_tensor(q))
    assert e.value.code == 1
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FspError):            # workspace too small
        F.rhs(cfg, Mg, Qg, ws=small)
    with pytest.raises(F.FspError):            # output aliasing the input
        F.rhs(cfg, Mg, Qg, out=Qg)


def test_full_size_riemann_1024_parity(F):
    # the 1024 x 1024 partially randomised Riemann grid at full size
    x, y = I.riemann_grid(1024, 0.3, 1811)
    q = I.riemann_quadrants(x, y)
    _check_case(F, _cfg(scheme=2, bc=(1, 1, 1, 1)), x, y, q)


def test_full_size_riemann_1024_rk3(F):
    """One TVD-RK3 step of the 1024 x 1024 Riemann grid at CFL 0.5 (the single-block
    workload at full size), FP64: the state and its change over the step."""
    x, y = I.riemann_grid(1024, 0.3, 1811)
    q = I.riemann_quadrants(x, y)
    cfgd = _cfg(scheme=2, bc=(1, 1, 1, 1))
    cfg = F.Config.from_dict(cfgd)
    M = O.metrics(cfgd, x, y)
    Mg, Q = _dev(M), _dev(q)
    ws = F.workspace(cfg, Q)
    dt = float(F.cfl_dt(cfg, Mg, Q, 0.5, ws=ws).item())
    assert abs(dt - O.cfl_dt(cfgd, M, q, 0.5)) < 1e-13 * dt
    F.rk3_step(cfg, Mg, Q, dt, ws=ws)
    q_o = O.rk3(cfgd, M, q, dt, 1)
    assert _rel(_host(Q) - q, q_o - q) < 1e-11
    assert _rel(_host(Q), q_o) < TOL_RHS


@pytest.mark.parametrize("shape", [(9, 2 * 65535), (8 * 65535, 9)])
def test_rhs_parity_longest_lines(F, shape):
    # the largest line counts the sweep grids allow (65535 CTAs across the lines of the xi
    # sweep, 2 rows each, and of the eta sweep, 8 columns each), transmissive faces
    ni, nj = shape
    h = 1.0 / 64
    x = np.broadcast_to(h * np.arange(ni, dtype=np.float64)[None, :], (nj, ni)).copy()
    y = np.broadcast_to(0.7 * h * np.arange(nj, dtype=np.float64)[:, None], (nj, ni)).copy()
    x, y = I.randomize(x, y, h, 0.7 * h, np.full((nj, ni), 0.2), seed=12)
    q = I.random_state((nj, ni), seed=13)
    _check_case(F, _cfg(scheme=2, bc=(1, 1, 1, 1)), x, y, q)
