"""fsp_rhs_noalloc, the right-hand side for callers that cannot allocate device memory
(for example a plugin inside an application that owns all device allocations): its
scratch is a fixed array inside the library.  Called through the C ABI, twice in a row on
different states, it must match fsp_rhs (which takes a caller-allocated workspace) within
the parity tolerance of the other GPU tests; a block too large for the array is refused."""
import numpy as np
import pytest

from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-12


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    fsp.lib()
    return fsp


def _noalloc(F, cfg, M, Q, out):
    # the binding's argument list for fsp_rhs_noalloc is declared with the others in fsp.py
    return F.rhs_noalloc_status(cfg, M, Q, out)


def test_noalloc_matches_rhs_twice_in_a_row(F):
    dev = torch.device("cuda")
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    cfg = F.Config(scheme=2, period=per)
    M = F.metrics(cfg, torch.as_tensor(x, device=dev), torch.as_tensor(y, device=dev))
    # the second state has smaller line maxima than the first: stale maxima left in the
    # shared array would change the second result
    qa = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 2.0, 1.5, 1.0), period=(10.0, 10.0))
    qb = I.isentropic_vortex(x, y, (3.0, 6.0), strength=2.0, free=(1.0, 0.2, 0.1, 1.0), period=(10.0, 10.0))
    for q in (qa, qb):
        Q = torch.as_tensor(q, device=dev)
        ref = F.rhs(cfg, M, Q)
        out = torch.full_like(Q, float("nan"))
        assert _noalloc(F, cfg, M, Q, out) == 0
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(o).all()
        assert np.abs(o - r).max() <= TOL_RHS * np.abs(r).max()


def test_noalloc_refuses_blocks_beyond_its_array(F):
    dev = torch.device("cuda")
    n = 1024   # 4 x 1024 x 1024 doubles of accumulator = 32 MiB > 8 MiB
    cfg = F.Config(scheme=2, period=((10.0, 0.0), (0.0, 10.0)))
    Q = torch.ones((4, n, n), dtype=torch.float64, device=dev)
    M = torch.ones((5, n + 8, n + 8), dtype=torch.float64, device=dev)
    out = torch.zeros_like(Q)
    assert _noalloc(F, cfg, M, Q, out) == 6          # FSP_ERR_NOMEM, nothing enqueued
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
