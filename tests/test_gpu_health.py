"""Failure detection on the GPU: fsp_check_state names the first node whose state is not finite
or not physical.  The failures are injected on the host (a NaN, a negative density, a negative
pressure written into the state before it is copied to the device); no kernel faults."""
import numpy as np
import pytest

from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


@pytest.mark.parametrize("prec", [0, 1])
def test_check_state_finds_the_first_bad_node(F, prec):
    ni, nj = 64, 40
    x, y, per = I.periodic_square(ni, 10.0, 0.2, seed=3, nj=nj)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=4.0, free=(1.0, 0.5, 0.2, 1.0), period=(10.0, 10.0))
    cfg = F.Config(scheme=2, period=per, precision=prec)
    dt = torch.float64 if prec == 0 else torch.float32
    Q = torch.as_tensor(q, dtype=dt, device="cuda")
    assert F.check_state(cfg, Q) == -1
    F.raise_on_bad(cfg, Q)                            # a valid state passes
    bad = q.copy()
    bad[1, 20, 33] = np.nan                           # non-finite momentum
    bad[3, 30, 5] = 0.1 * bad[3, 30, 5] - 5.0         # energy below the kinetic energy: p < 0
    bad[0, 35, 60] = -bad[0, 35, 60]                  # negative density
    Qb = torch.as_tensor(bad, dtype=dt, device="cuda")
    assert F.check_state(cfg, Qb) == 20 * ni + 33
    Qb[1, 20, 33] = Q[1, 20, 33]
    assert F.check_state(cfg, Qb) == 30 * ni + 5
    Qb[3, 30, 5] = Q[3, 30, 5]
    with pytest.raises(F.FspError) as e:
        F.raise_on_bad(cfg, Qb)
    assert e.value.code == 4 and e.value.node == (35, 60)
