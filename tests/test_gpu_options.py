"""The options beyond the paper's tested schemes on the GPU against the oracle (Section 7 names
them as further directions; the free parameter is that of Eqs. 3.5 and 3.17 and of the
Appendix's scheme (1)): WENO-Z weights (weights = 1), Steger-Warming and Van Leer splitting of
the midpoint flux (mid_split = 1, 2), and the one-midpoint schemes at a free parameter
alpha != 1 (scheme_alpha), with the metrics from that scheme's own central operator.

The oracle's options are pinned on the CPU (the options' test module there).  Bars as for the
printed schemes: FP64 relative max-norm <= 1e-12 for metrics, right-hand sides and RK3
states; FP32 and mixed precision against the FP64 oracle on the float-rounded state <= 1e-4
and 5e-5.  The tile kernels run the options (the marching passes are compiled for the
printed schemes only and are refused for the options); the adjoint refuses them too."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
BOUND = {1: 1e-4, 2: 5e-5}
GAMMA = 1.4

OPTIONS = [dict(weights=1), dict(mid_split=1), dict(mid_split=2), dict(scheme_alpha=1.3),
           dict(scheme_alpha=0.7), dict(weights=1, mid_split=2, scheme_alpha=1.2)]


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


def _applies(scheme, opt):
    # the free parameter belongs to the one-midpoint schemes
    return opt.get("scheme_alpha", 1.0) == 1.0 or scheme in (0, 2, 4)


def _ragged(ni=97, nj=41, seed=8):
    x, y, per = I.periodic_square(ni, 12.0, 0.2, seed=seed, nj=nj)
    q = I.isentropic_vortex(x, y, (6.0, 6.0), strength=4.0, free=(1.0, 0.7, -0.4, 1.0), period=(12.0, 12.0))
    return x, y, per, q


def _check(F, cfgd, x, y, q):
    cfg = F.Config.from_dict(cfgd)
    M_o = O.metrics(cfgd, x, y)
    Mh = _host(F.metrics(cfg, _dev(x), _dev(y)))
    assert _rel(Mh[:4], M_o[:4]) < TOL and _rel(Mh[4], M_o[4]) < TOL
    R_o = O.rhs(cfgd, M_o, q)
    err = _rel(_host(F.rhs(cfg, _dev(M_o), _dev(q))), R_o)
    assert err < TOL, (cfgd, err)
    return err


@pytest.mark.parametrize("opt", OPTIONS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_options_rhs_parity_ragged_tiles(F, scheme, opt):
    if not _applies(scheme, opt):
        pytest.skip("the free parameter belongs to the one-midpoint schemes")
    x, y, per, q = _ragged()
    _check(F, dict(scheme=scheme, period=per, **opt), x, y, q)


@pytest.mark.parametrize("opt", OPTIONS[:3], ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_options_rhs_parity_riemann_and_boundaries(F, opt):
    """Shocks and slip lines: the splittings' branches and the WENO-Z weights at
    discontinuities (transmissive faces), and every boundary kind on a random state.  The
    splittings need the sound speed of the reconstructed midpoint states: with the Riemann
    quadrants against the fixed face states of Dirichlet or far-field faces, WENOIU3's
    reconstruction next to the low-pressure quadrant has negative pressure and the oracle's
    right-hand side is NaN there as well, so that pairing is not a case."""
    x, y = I.riemann_grid(60, 0.3, 1811)
    st = np.stack([I.conservative(1.0, 0.8, 0.3, 1.0 / GAMMA), I.conservative(1.1, 0.7, 0.2, 0.8),
                   I.conservative(0.9, -0.5, 0.1, 0.75), I.conservative(1.05, 0.6, -0.3, 0.7)])
    for bc, q in [((1, 1, 1, 1), I.riemann_quadrants(x, y)), ((2, 3, 4, 1), I.random_state(x.shape, seed=32))]:
        for scheme in (0, 3, 4):
            _check(F, dict(scheme=scheme, bc=bc, bc_state=st, **opt), x, y, q)


def test_options_supersonic_stream(F):
    """A Mach 3 stream at an angle: Van Leer's and Steger-Warming's fully upwind branches on
    every interface of one direction."""
    x, y, per = I.periodic_square(48, 8.0, 0.2, seed=4)
    q = I.isentropic_vortex(x, y, (4.0, 4.0), strength=2.0, free=(1.0, 3.0, 0.8, 0.7), period=(8.0, 8.0))
    for split in (1, 2):
        _check(F, dict(scheme=2, period=per, mid_split=split), x, y, q)


@pytest.mark.parametrize("opt", [dict(weights=1), dict(mid_split=2), dict(scheme_alpha=1.3)],
                         ids=["weno_z", "van_leer", "alpha"])
def test_options_rk3_and_free_stream(F, opt):
    x, y, per = I.periodic_square(64, 8.0, 0.2, seed=21, nj=40)
    q = I.random_state(x.shape, seed=33)
    cfgd = dict(scheme=2, period=per, **opt)
    cfg = F.Config.from_dict(cfgd)
    M = O.metrics(cfgd, x, y)
    q_o = O.rk3(cfgd, M, q, 0.01, 2)
    Q = _dev(q)
    for _ in range(2):
        F.rk3_step(cfg, _dev(M), Q, 0.01)
    assert _rel(_host(Q), q_o) < TOL
    # free stream on the randomised grid, with the metrics of the scheme's own operator
    Mg = F.metrics(cfg, _dev(x), _dev(y))
    q0 = _dev(I.uniform_state(x.shape, 1.0, 0.5, 0.3, 1.0 / GAMMA))
    assert float(F.rhs(cfg, Mg, q0).abs().max()) < 1e-12


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("opt", OPTIONS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_options_float_paths(F, prec, opt):
    if prec == 2 and opt.get("mid_split", 0):
        pytest.skip("the splittings are refused in mixed precision (checked below)")
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    q32 = q.astype(np.float32).astype(np.float64)
    for scheme in (0, 2, 4):
        cfgd = dict(scheme=scheme, period=per, **opt)
        M = O.metrics(cfgd, x, y)
        R = O.rhs(cfgd, M, q32)
        cfg = F.Config.from_dict(dict(cfgd, precision=prec))
        Rg = F.rhs(cfg, _dev(M), _dev(q32, torch.float32))
        assert Rg.dtype == torch.float32
        assert _rel(_host(Rg), R) < BOUND[prec], (scheme, prec, opt)


def test_options_refusals(F):
    x, y, per, q = _ragged(40, 24)
    M, Q = _dev(O.metrics(dict(scheme=2, period=per), x, y)), _dev(q)
    refused = [dict(scheme=2, mid_split=1, precision=2),       # splitting: same precision only
               dict(scheme=1, scheme_alpha=1.3),                # two-midpoint: no free parameter
               dict(scheme=2, weights=2), dict(scheme=2, mid_split=3), dict(scheme=2, scheme_alpha=-1.0)]
    for cfgd in refused:
        cfg = F.Config.from_dict(dict(cfgd, period=per))
        with pytest.raises(F.FspError):
            F.rhs(cfg, M, Q.float() if cfgd.get("precision") else Q)     # metrics stay FP64
    # the adjoint is the printed schemes' only
    cfg = F.Config.from_dict(dict(scheme=2, period=per, weights=1))
    with pytest.raises(F.FspError) as e:
        F.rhs_vjp(cfg, M, Q, torch.ones_like(Q))
    assert e.value.code == 2


def _small_cylinder():
    return I.cylinder_blocks(imin=24, imax=48, jmin=16, jmax=32, step=8, cols=4, rows=3, stretch=1.02,
                             frac_random=0.5)


@pytest.mark.parametrize("opt", [dict(weights=1), dict(mid_split=1), dict(scheme_alpha=1.3)],
                         ids=["weno_z", "steger_warming", "alpha"])
def test_options_batch_tiles(F, opt):
    """The multi-block batch with every tile shape; the marching shape is refused."""
    blocks, states, free = _small_cylinder()
    rng = np.random.default_rng(5)
    qs = []
    for q in states:
        rho = q[0] * (1 + 0.05 * rng.standard_normal(q[0].shape))
        u = q[1] / q[0] + 0.05 * rng.standard_normal(q[0].shape)
        v = q[2] / q[0] + 0.05 * rng.standard_normal(q[0].shape)
        p = 0.4 * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0])
        qs.append(I.conservative(rho, u, v, p))
    cfgd = dict(scheme=2, bc_state=np.tile(free, (4, 1)), **opt)
    Ms = O.mb_metrics(cfgd, blocks)
    Ro = O.mb_rhs(cfgd, blocks, Ms, qs)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, qs)
    Mg = [m.cpu().numpy() for m in bt.metrics()]
    assert max(np.abs(a - b).max() for a, b in zip(Mg, Ms)) < TOL * max(np.abs(b).max() for b in Ms)
    for k in range(len(blocks)):
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    scale = max(np.abs(r).max() for r in Ro)
    for v in (0, 1, 2):
        bt.set_tile_shape(0, v)
        bt.set_tile_shape(1, v)
        Rg = [r.cpu().numpy() for r in bt.rhs()]
        assert max(np.abs(a - b).max() for a, b in zip(Rg, Ro)) < TOL * scale, v
    with pytest.raises(F.FspError) as e:
        bt.set_tile_shape(0, 3)
    assert e.value.code == 2
    bt.close()
