"""FP32 paths against the FP64 oracle (same seeded inputs, the state rounded to float first).

Stated bounds (relative max-norm of the right-hand side against the FP64 oracle):
* FSP_FP32 (everything in float):                      <= 1e-4
* FSP_FP32_MIXED (WENO in float, fluxes/h in double):   <= 5e-5
Measured on GB300: at most 3.8e-5 (FP32) and 2.2e-5 (mixed) on the 256 x 256 vortex, where the
right-hand side is a small difference of O(1) fluxes, and below 2e-7 on the Riemann grid.
Free stream: the mixed path keeps the FP64 residual (metric products and differences in
double); the plain FP32 path's residual is at FP32 round-off."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BOUND = {1: 1e-4, 2: 5e-5}
GAMMA = 1.4


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _run(F, cfgd, x, y, q, prec):
    M = O.metrics(cfgd, x, y)
    q32 = q.astype(np.float32).astype(np.float64)
    R = O.rhs(cfgd, M, q32)
    cfg = F.Config.from_dict(dict(cfgd, precision=prec))
    Rg = F.rhs(cfg, torch.as_tensor(M, device="cuda"), torch.as_tensor(q32, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert Rg.dtype == torch.float32
    return _rel(Rg.double().cpu().numpy(), R)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_fp32_rhs_vortex_256(F, prec, scheme):
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    assert _run(F, dict(scheme=scheme, period=per), x, y, q, prec) < BOUND[prec]


@pytest.mark.parametrize("prec", [1, 2])
def test_fp32_rhs_riemann_and_boundaries(F, prec):
    x, y = I.riemann_grid(96, 0.3, 1811)
    q = I.riemann_quadrants(x, y)
    # a different state on every face, so that each face must read its own
    st = np.stack([I.conservative(1.0, 0.8, 0.3, 1.0 / GAMMA), I.conservative(1.1, 0.7, 0.2, 0.8),
                   I.conservative(0.9, -0.5, 0.1, 0.75), I.conservative(1.05, 0.6, -0.3, 0.7)])
    for bc in [(1, 1, 1, 1), (2, 3, 4, 1), (4, 2, 2, 4)]:
        for scheme in (0, 3):
            assert _run(F, dict(scheme=scheme, bc=bc, bc_state=st), x, y, q, prec) < BOUND[prec]


def test_free_stream_fp32_paths(F):
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q0 = np.array([1.0, 1.0, 1.0, 1.0 / (GAMMA - 1) + 1.0])
    for scheme in range(5):
        cfgd = dict(scheme=scheme, period=per)
        r64 = O.fsp_residual(cfgd, x, y, q0)
        for prec in (1, 2):
            cfg = F.Config.from_dict(dict(cfgd, precision=prec))
            Mg = F.metrics(cfg, torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"))
            Q = torch.as_tensor(I.uniform_state(x.shape, 1.0, 1.0, 1.0, 1.0), dtype=torch.float32, device="cuda")
            r = float(F.rhs(cfg, Mg, Q).abs().max())
            if prec == 2:
                assert r < 4 * r64 + 1e-14      # FP64 round-off
            else:
                assert r < 1e-3                 # FP32 round-off at h = 10/256


def test_fp32_rk3_steps(F):
    x, y, per = I.periodic_square(96, 8.0, 0.2, seed=6)
    q = I.isentropic_vortex(x, y, (4.0, 4.0), strength=4.0, free=(1.0, 0.7, -0.4, 1.0), period=(8.0, 8.0))
    cfgd = dict(scheme=2, period=per)
    M = O.metrics(cfgd, x, y)
    q32 = q.astype(np.float32).astype(np.float64)
    dt = 0.5 * O.cfl_dt(cfgd, M, q32, 1.0)
    q_o = O.rk3(cfgd, M, q32, dt, 3)
    for prec in (1, 2):
        cfg = F.Config.from_dict(dict(cfgd, precision=prec))
        Qg = torch.as_tensor(q32, dtype=torch.float32, device="cuda")
        Mg = torch.as_tensor(M, device="cuda")
        ws = F.workspace(cfg, Qg)
        for _ in range(3):
            F.rk3_step(cfg, Mg, Qg, dt, ws=ws)
        torch.cuda.synchronize()
        change = Qg.double().cpu().numpy() - q32
        assert _rel(change, q_o - q32) < 1e-3     # the update itself, not the rounded state
