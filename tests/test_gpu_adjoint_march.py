"""The autograd layer over the adjoint: torch.autograd.gradcheck of FspRHS and FspMetrics;
the gradient of a march of RK3 steps with checkpointing against the oracle's exact
forward-mode tangent on small and full-size shock-vortex cases; and the full shock-vortex
gradient (512 x 512, 200 steps at CFL 0.5, checkpoint every 14 steps) against fourth-order
central finite differences on smooth random directions and on single nodes."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I
from paper_1810_11103_gb300 import objectives as J

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


@pytest.fixture(scope="module")
def A(F):
    from paper_1810_11103_gb300 import autograd
    return autograd


def _dev(a, grad=False):
    t = torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    return t.requires_grad_(grad)


def _sv_cfgd(eps=1e-6):
    bc, st = I.shock_vortex_bc()
    return dict(scheme=2, bc=bc, bc_state=st, eps=eps)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (3, 3, 1, 2)])
def test_gradcheck_rhs(F, A, bc):
    if bc[0] == 0:
        x, y, per = I.periodic_square(12, 6.0, 0.2, seed=4, nj=10)
    else:
        x, y = I.riemann_grid(12, 0.2, 8)
        x, y = x[:10], y[:10] * 1.2
        per = ((0.0, 0.0), (0.0, 0.0))
    st = np.tile(I.conservative(1.0, 0.3, 0.1, 0.8), (4, 1))
    cfg = F.Config.from_dict(dict(scheme=3, bc=bc, bc_state=st, period=per))
    M = F.metrics(cfg, _dev(x), _dev(y)).detach().requires_grad_(True)
    Q = _dev(I.random_state(x.shape, seed=44), True)
    assert torch.autograd.gradcheck(lambda m, q: A.rhs(cfg, m, q), (M, Q), eps=1e-6, atol=1e-6, rtol=1e-5,
                                    nondet_tol=1e-12)


def test_gradcheck_metrics(F, A):
    x, y = I.riemann_grid(12, 0.25, 9)
    cfg = F.Config.from_dict(dict(scheme=2, bc=(1, 1, 3, 3)))
    assert torch.autograd.gradcheck(lambda a, b: A.metrics(cfg, a, b), (_dev(x, True), _dev(y, True)),
                                    eps=1e-6, atol=1e-6, rtol=1e-5, nondet_tol=1e-12)


def _oracle_march(cfgd, x, y, q0, nsteps, cfl):
    """Oracle states and CFL time steps of the march (the steps are oracle outputs)."""
    M = O.metrics(cfgd, x, y)
    q, dts = q0.copy(), []
    for _ in range(nsteps):
        dts.append(O.cfl_dt(cfgd, M, q, cfl))
        q = O.rk3(cfgd, M, q, dts[-1], 1)
    return M, q, dts


@pytest.mark.parametrize("every", [5, 0])
def test_march_gradient_vs_oracle_tangent(F, A, every):
    x, y = I.shock_vortex_grid(48, 40, beta=2.0)
    q0 = I.shock_vortex_state(x, y)
    cfgd = _sv_cfgd()
    M, qN, dts = _oracle_march(cfgd, x, y, q0, 16, 0.5)
    win = J.window_of(x)
    # directional derivative by the oracle's tangent along smooth random directions
    dq0 = np.stack([0.01 * I.smooth_field(x.shape, 100 + v) for v in range(4)])
    dx = 0.002 * I.smooth_field(x.shape, 200)
    dy = 0.002 * I.smooth_field(x.shape, 201)
    Mo, dM = O.metrics_jvp(cfgd, x, y, dx, dy)
    q, dq = q0.copy(), dq0.copy()
    for dt in dts:
        q, dq = O.rk3_jvp(cfgd, Mo, q, dq, dt, 1, dM)
    tq, tx, ty, tm = (torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (q, x, y, Mo))
    J.shock_vortex_functional(tq, tx, ty, tm, win).backward()
    d_oracle = float((tq.grad.numpy() * dq).sum() + (tx.grad.numpy() * dx).sum() + (ty.grad.numpy() * dy).sum()
                     + (tm.grad.numpy() * dM).sum())
    # the same by the GPU adjoint through autograd
    cfg = F.Config.from_dict(cfgd)
    gx, gy, gq = _dev(x, True), _dev(y, True), _dev(q0, True)
    Mg = A.metrics(cfg, gx, gy)
    QN = A.rk3_march(cfg, Mg, gq, dts, every)
    assert np.abs(QN.detach().cpu().numpy() - qN).max() < 1e-12 * np.abs(qN).max()
    J.shock_vortex_functional(QN, gx, gy, Mg, win).backward()
    d_gpu = float((gq.grad.cpu().numpy() * dq0).sum() + (gx.grad.cpu().numpy() * dx).sum()
                  + (gy.grad.cpu().numpy() * dy).sum())
    assert abs(d_gpu - d_oracle) < 1e-9 * abs(d_oracle), (d_gpu, d_oracle)


def test_shock_vortex_512_gradient_vs_finite_differences(F, A):
    x, y = I.shock_vortex_grid(512)
    q0 = I.shock_vortex_state(x, y)
    cfgd = _sv_cfgd()
    cfg = F.Config.from_dict(cfgd)
    win = J.window_of(x)
    gx, gy, gq = _dev(x, True), _dev(y, True), _dev(q0, True)
    with torch.no_grad():
        dts, _ = A.cfl_schedule(cfg, F.metrics(cfg, gx, gy), gq, 200, 0.5)
    Mg = A.metrics(cfg, gx, gy)
    QN = A.rk3_march(cfg, Mg, gq, dts, 14)
    J.shock_vortex_functional(QN, gx, gy, Mg, win).backward()
    grad_q, grad_x, grad_y = gq.grad.double(), gx.grad.double(), gy.grad.double()

    @torch.no_grad()
    def terms(dq, dx, dy):
        xx, yy = gx.detach() + dx, gy.detach() + dy
        M = F.metrics(cfg, xx, yy)
        Q = gq.detach() + dq
        ws = F.workspace(cfg, Q)
        for dt in dts:
            F.rk3_step(cfg, M, Q, dt, ws=ws)
        return J.terms(Q, xx, yy, M, win)

    def fd(dq, dx, dy, h):
        """Fourth-order central difference (8 (J(h) - J(-h)) - (J(2h) - J(-2h))) / 12h, each
        difference taken node by node before the sum.  Its h^2 term cancels, which matters
        where a single-node kick meets nearly uniform data: there the nonlinear weights bend
        on the scale h^2 / epsilon."""
        out = 0.0
        for c, s in ((8.0, 1.0), (-1.0, 2.0)):
            bp, wp = terms(s * h * dq, s * h * dx, s * h * dy)
            bm, wm = terms(-s * h * dq, -s * h * dx, -s * h * dy)
            out += c * float((bp - bm).sum() + (wp - wm).sum())
        return out / (12.0 * h)

    nj, ni = x.shape
    i0, i1 = win
    zq, zc = torch.zeros_like(gq), torch.zeros_like(gx)
    dirs = []
    for v in range(4):                         # smooth state directions
        dq = torch.stack([_dev(I.smooth_field(x.shape, 300 + 4 * v + c)) * s
                          for c, s in enumerate((1.0, 1.0, 1.0, 2.0))])
        dirs.append(("state", dq, zc, zc))
    for v in range(4):                         # smooth grid directions (0.1 of the finest spacing)
        dirs.append(("grid", zq, _dev(0.004 * I.smooth_field(x.shape, 400 + v)),
                     _dev(0.004 * I.smooth_field(x.shape, 410 + v))))
    # Single nodes, each with its step fixed by where it sits.  The error of the difference is
    # V-shaped in h: where the kick meets exactly uniform data (the inflow ahead of the shock,
    # and behind it) the weights bend on the scale h^2/epsilon, so a small step; where its
    # domain of influence reaches the shock and the vortex inside the window, the differences
    # of J carry a rounding floor of about 1e-14 after 200 steps, so a large one.
    nodes = [((0, nj // 2, (i0 + i1) // 2), 1e-4),     # window centre: shock and vortex
             ((3, nj // 2 + 5, i0 + 3), 1e-4),         # window edge, next to the shock
             ((1, nj // 3, 2), 1e-5),                  # uniform inflow
             ((2, nj // 2 + 2, ni - ni // 4), 1e-5)]   # uniform flow behind the shock
    for (c, j, i), h in nodes:
        dq = torch.zeros_like(gq)
        dq[c, j, i] = 1.0
        dirs.append(("state node", dq, zc, zc, h))
    for name, dq, dx, dy, *hs in dirs:
        adj = float((grad_q * dq).sum() + (grad_x * dx).sum() + (grad_y * dy).sum())
        # Steps.  Whole-field state kicks: 1e-7 (larger ones start to switch the argmax of
        # nearly tied line maxima of the spectral radius, a kink).  Grid directions: 1e-5
        # (the metrics difference coordinates of size 10 at spacings of 0.04, so smaller
        # steps drown in their rounding).
        h = hs[0] if hs else {"state": 1e-7, "grid": 1e-5}[name]
        num = fd(dq, dx, dy, h)
        rel = abs(adj - num) / abs(num)
        print(f"{name}: h {h:.0e} adjoint {adj:.12e} finite difference {num:.12e} relative {rel:.2e}")
        assert rel < 1e-6, (name, adj, num, rel)
    # Single grid nodes where the flow is uniform (the outflow face, the region behind the
    # shock) have zero derivative: a uniform flow stays uniform on any grid (free-stream
    # preservation), the window sum of J^-1 telescopes to its edges, and the arc length of
    # the straight outflow face is unchanged to first order under uniform pressure.
    scale = float(torch.maximum(grad_x.abs().max(), grad_y.abs().max()))
    for (j, i, which) in [(nj // 2, 0, 0), (nj // 4, 0, 1), (nj // 2 - 40, i0 + 30, 0), (nj // 2 + 60, i0 + 20, 1)]:
        d = torch.zeros_like(gx)
        d[j, i] = 1.0
        adj = float((grad_y if which else grad_x)[j, i])
        num = fd(zq, zc if which else d, d if which else zc, 1e-4)
        print(f"uniform-flow grid node ({j}, {i}): adjoint {adj:.3e} finite difference {num:.3e} "
              f"(largest nodal grid derivative {scale:.3e})")
        assert abs(adj) < 1e-6 * scale and abs(num) < 1e-6 * scale, (j, i, adj, num, scale)


def test_shock_vortex_512_gradient_vs_oracle_tangent(F, A):
    # Full size (many tiles along both directions), a few steps: the oracle's exact tangent
    # along one direction mixing single-node kicks with smooth state and grid directions.
    # The grid-node kick sits in the vortex, where finite differences cannot check it: as
    # the vortex moves, the argmax of the line maxima of the spectral radius hops from node
    # to node, and J, a function of that node's coordinate, has kinks spaced below 1e-5.
    x, y = I.shock_vortex_grid(512)
    q0 = I.shock_vortex_state(x, y)
    cfgd = _sv_cfgd()
    M, _, dts = _oracle_march(cfgd, x, y, q0, 6, 0.5)
    win = J.window_of(x)
    nj, ni = x.shape
    dq0 = np.stack([0.01 * I.smooth_field(x.shape, 500 + v) for v in range(4)])
    dq0[0, nj // 2, (win[0] + win[1]) // 2] += 1.0
    dx, dy = 0.004 * I.smooth_field(x.shape, 510), 0.004 * I.smooth_field(x.shape, 511)
    dy[nj // 2 + 10, ni - ni // 4] += 0.05
    Mo, dM = O.metrics_jvp(cfgd, x, y, dx, dy)
    q, dq = q0.copy(), dq0.copy()
    for dt in dts:
        q, dq = O.rk3_jvp(cfgd, Mo, q, dq, dt, 1, dM)
    tq, tx, ty, tm = (torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (q, x, y, Mo))
    J.shock_vortex_functional(tq, tx, ty, tm, win).backward()
    d_oracle = float((tq.grad.numpy() * dq).sum() + (tx.grad.numpy() * dx).sum() + (ty.grad.numpy() * dy).sum()
                     + (tm.grad.numpy() * dM).sum())
    cfg = F.Config.from_dict(cfgd)
    gx, gy, gq = _dev(x, True), _dev(y, True), _dev(q0, True)
    Mg = A.metrics(cfg, gx, gy)
    QN = A.rk3_march(cfg, Mg, gq, dts, 4)
    J.shock_vortex_functional(QN, gx, gy, Mg, win).backward()
    d_gpu = float((gq.grad.cpu().numpy() * dq0).sum() + (gx.grad.cpu().numpy() * dx).sum()
                  + (gy.grad.cpu().numpy() * dy).sum())
    assert abs(d_gpu - d_oracle) < 1e-10 * abs(d_oracle), (d_gpu, d_oracle)
