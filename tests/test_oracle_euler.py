"""Pins of the oracle's 2-D Euler right-hand side against what the paper and the
mathematics fix (CPU only): exact metrics on affine and polynomial grids, free-stream
preservation (Section 5.2, Table 4) with a negative control, telescoping conservation,
mirror and transpose symmetry, reduction to the closed-form linear upwind operator,
design order on a curved grid, line spectral radius and time step in closed form, the
RK3 order in time, and the Sod tube against the exact Riemann solution.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

G = O.G
GAMMA = 1.4


def _cfg(**kw):
    c = dict(scheme=2, interp=0, ppm=1, linear_weights=0, bc=(0, 0, 0, 0), gamma=GAMMA,
             lf_alpha=1.1, eps=1e-40, period=((0.0, 0.0), (0.0, 0.0)))
    c.update(kw)
    return c


def _affine(ni, nj, h=0.5, s=0.2, periodic=True):
    i = np.arange(ni, dtype=float)
    j = np.arange(nj, dtype=float)
    X = h * i[None, :] + s * j[:, None]
    Y = h * j[:, None] + 0.0 * i[None, :]
    per = ((ni * h, 0.0), (nj * s, nj * h))
    return X, Y, per


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("periodic", [True, False])
def test_metrics_exact_on_affine_grid(scheme, periodic):
    ni, nj, h, s = 12, 11, 0.5, 0.2
    x, y, per = _affine(ni, nj, h, s)
    bc = (0, 0, 0, 0) if periodic else (1, 1, 1, 1)
    M = O.metrics(_cfg(scheme=scheme, period=per, bc=bc), x, y)
    # x_xi = h, x_eta = s, y_xi = 0, y_eta = h at every node, ghosts included
    for p, want in enumerate([h, -s, 0.0, h, h * h]):
        assert np.allclose(M[p], want, atol=1e-13), p


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_metrics_exact_on_polynomial_grid(scheme):
    # a curved, non-periodic grid whose coordinates are polynomials of degree <= 4 (third
    # order schemes), 6 (fifth order) or 8 (seventh): the central operators differentiate
    # them exactly
    deg = 4 if scheme < 2 else 6 if scheme < 4 else 8
    n = 30
    s = np.arange(n, dtype=float) / n
    XI, ETA = np.meshgrid(s, s)
    x = XI + 0.3 * ETA ** (deg - 1) + 0.1 * XI ** deg
    y = ETA + 0.2 * XI ** (deg - 1) * 1.0 + 0.05 * ETA ** deg
    M = O.metrics(_cfg(scheme=scheme, bc=(1, 1, 1, 1)), x, y)
    x_xi = (1.0 + 0.1 * deg * XI ** (deg - 1)) / n
    x_eta = 0.3 * (deg - 1) * ETA ** (deg - 2) / n
    y_xi = 0.2 * (deg - 1) * XI ** (deg - 2) / n
    y_eta = (1.0 + 0.05 * deg * ETA ** (deg - 1)) / n
    core = (slice(8, n - 8), slice(8, n - 8))   # away from the reflected ghosts
    inner = lambda A: A[G:-G, G:-G][core]
    assert np.allclose(inner(M[0]), y_eta[core], atol=1e-13)
    assert np.allclose(inner(M[1]), -x_eta[core], atol=1e-13)
    assert np.allclose(inner(M[2]), -y_xi[core], atol=1e-13)
    assert np.allclose(inner(M[3]), x_xi[core], atol=1e-13)
    assert np.allclose(inner(M[4]), (x_xi * y_eta - x_eta * y_xi)[core], atol=1e-13)


def _uniform_q(u=1.0, v=1.0, rho=1.0, p=1.0):
    return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("interp", [0, 1])
def test_free_stream_preservation_randomized_grid(scheme, interp):
    x, y, per = I.periodic_square(32, 10.0, 0.2, seed=1810)
    cfg = _cfg(scheme=scheme, interp=interp, period=per)
    q0 = _uniform_q(1.0, 1.0, 1.0, 1.0)
    r64 = O.fsp_residual(cfg, x, y, q0)
    assert r64 < 2e-12
    # computed in a wider type the residual shrinks with the precision: it is round-off
    if O.long_double_digits() > 53:
        rwide = O.fsp_residual(cfg, x, y, q0, wide=True)
        assert rwide < r64 * 2.0 ** (53 - O.long_double_digits()) * 64


def test_free_stream_negative_controls():
    x, y, per = I.periodic_square(32, 10.0, 0.2, seed=1810)
    q = I.uniform_state(x.shape, 1.0, 1.0, 1.0, 1.0)
    # metrics with the fourth-order operator of WENOIU3-1MP but fluxes of WENOIU5-1MP
    M_wrong = O.metrics(_cfg(scheme=0, period=per), x, y)
    assert np.abs(O.rhs(_cfg(scheme=2, period=per), M_wrong, q)).max() > 1e-4
    # metric midpoint interpolation differing between metrics and fluxes
    M_avg = O.metrics(_cfg(scheme=2, interp=1, period=per), x, y)
    assert np.abs(O.rhs(_cfg(scheme=2, interp=0, period=per), M_avg, q)).max() > 1e-4


def _table4():
    path = os.path.join(os.path.dirname(__file__), "golden", "table4.csv")
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    return [float(r.split(",")[1]) for r in rows]


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_table4_free_stream_on_paper_grid(scheme):
    # Section 5.2: uniform Mach 0.5 flow on the 81 x 81 randomised grid (L = 16, A = 0.45),
    # dt = 0.01.  The paper runs 1000 steps; 20 steps keep the CPU suite short.
    x, y = I.paper_random_grid(81, 81, 16.0, 0.45, seed=1810)
    cfg = _cfg(scheme=scheme, bc=(1, 1, 1, 1))
    M = O.metrics(cfg, x, y)
    c = 1.0
    q = I.uniform_state(x.shape, 1.0, 0.5 * c, 0.0, 1.0 / GAMMA)
    q = O.rk3(cfg, M, q, 0.01, 20)
    v = q[2] / q[0]
    l2 = math.sqrt((v * v).mean())
    assert l2 < 10 * _table4()[scheme]


def test_conservation_periodic():
    x, y, per = I.periodic_square(24, 6.0, 0.2, seed=11, nj=20)
    for scheme in range(5):
        cfg = _cfg(scheme=scheme, period=per)
        M = O.metrics(cfg, x, y)
        q = I.random_state(x.shape, seed=5)
        R = O.rhs(cfg, M, q)
        J = M[4, G:-G, G:-G]
        for v in range(4):
            s = (J * R[v]).sum()
            assert abs(s) < 1e-13 * np.abs(J * R[v]).sum(), (scheme, v, s)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_mirror_symmetry(scheme):
    ni = nj = 20
    x, y, per = I.periodic_square(ni, 8.0, 0.2, seed=3)
    q = I.isentropic_vortex(x, y, (4.3, 3.7), strength=4.0, free=(1.0, 0.3, -0.2, 1.0), period=(8.0, 8.0))
    cfg = _cfg(scheme=scheme, period=per)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    # reflect i -> ni-1-i, x -> -x, rho u -> -rho u
    xr, yr = -x[:, ::-1], y[:, ::-1].copy()
    qr = q[:, :, ::-1].copy()
    qr[1] *= -1
    Rr = O.rhs(cfg, O.metrics(cfg, xr, yr), qr)
    back = Rr[:, :, ::-1].copy()
    back[1] *= -1
    assert np.allclose(back, R, rtol=0, atol=1e-12 * np.abs(R).max())


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_transpose_symmetry(scheme):
    x, y, per = I.periodic_square(18, 8.0, 0.2, seed=4)
    q = I.isentropic_vortex(x, y, (4.3, 3.7), strength=4.0, free=(1.0, 0.3, -0.2, 1.0), period=(8.0, 8.0))
    cfg = _cfg(scheme=scheme, period=per)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    xt, yt = y.T.copy(), x.T.copy()
    qt = np.stack([q[0].T, q[2].T, q[1].T, q[3].T])
    Rt = O.rhs(cfg, O.metrics(cfg, xt, yt), qt)
    back = np.stack([Rt[0].T, Rt[2].T, Rt[1].T, Rt[3].T])
    assert np.allclose(back, R, rtol=0, atol=1e-12 * np.abs(R).max())


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_rotation_equivariance(scheme):
    """The Euler equations do not single out a direction.  The metric formulation (Section 2)
    and the characteristic projection along the averaged metric direction (Section 3.4)
    inherit that.  Rotating the grid, its periods and the velocity by a generic angle
    rotates the momentum components of the right-hand side and leaves density and energy
    alone.  A perturbed vortex makes the nonlinear weights matter, so a projection in any
    other direction, which is still exact for linear weights and uniform flow, breaks this."""
    x, y, per = I.periodic_square(20, 8.0, 0.2, seed=5)
    q = I.isentropic_vortex(x, y, (4.3, 3.7), strength=4.0, free=(1.0, 0.3, -0.2, 1.0), period=(8.0, 8.0))
    rng = np.random.default_rng(9)
    rho = q[0] * (1 + 0.1 * rng.standard_normal(q[0].shape))
    u = q[1] / q[0] + 0.1 * rng.standard_normal(q[0].shape)
    p = (GAMMA - 1) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0])
    q = I.conservative(rho, u, q[2] / q[0], p)
    cfg = _cfg(scheme=scheme, period=per)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    c, s = np.cos(0.5), np.sin(0.5)
    xr, yr = c * x - s * y, s * x + c * y
    cfgr = _cfg(scheme=scheme, period=tuple((c * a - s * b, s * a + c * b) for a, b in per))
    qr = q.copy()
    qr[1], qr[2] = c * q[1] - s * q[2], s * q[1] + c * q[2]
    Rr = O.rhs(cfgr, O.metrics(cfgr, xr, yr), qr)
    back = Rr.copy()
    back[1], back[2] = c * Rr[1] + s * Rr[2], -s * Rr[1] + c * Rr[2]
    assert np.abs(back - R).max() < 1e-11 * np.abs(R).max()


def _euler_x_flux(q, mx, my, gamma=GAMMA):
    rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
    p = (gamma - 1) * (q[3] - 0.5 * rho * (u * u + v * v))
    U = mx * u + my * v
    return np.stack([rho * U, rho * u * U + mx * p, rho * v * U + my * p, (q[3] + p) * U])


def _closed_form_linear_rhs(scheme, q, h, alpha=1.1, gamma=GAMMA):
    """The linear upwind operator on a uniform Cartesian periodic grid written directly:
    with omega_k = C_k the characteristic interpolation reduces to the linear midpoint
    interpolation of Q itself (Table 1 combined with its C_k)."""
    tab = O.scheme_table(scheme)
    r = tab["r"]
    total = np.zeros_like(q)
    for axis, (mx, my) in ((2, (h, 0.0)), (1, (0.0, h))):
        sh = lambda a, k: np.roll(a, -k, axis=axis)    # value at index + k
        rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
        p = (gamma - 1) * (q[3] - 0.5 * rho * (u * u + v * v))
        c = np.sqrt(gamma * p / rho)
        sp = np.abs(mx * u + my * v) + c * math.hypot(mx, my)
        A = alpha * (sp.max(axis=1, keepdims=True) if axis == 2 else sp.max(axis=0, keepdims=True))
        if r == 4:
            # the 7-point interpolant at j + 1/2 (nodes j-3 .. j+3), and its mirror
            cs = np.array([-5, 42, -175, 700, 525, -70, 7]) / 1024
            lin = lambda a: sum(c * sh(a, m) for c, m in zip(cs, range(-3, 4)))
            linm = lambda a: sum(c * sh(a, 1 - m) for c, m in zip(cs, range(-3, 4)))
        elif r == 3:
            lin = lambda a: (3 * sh(a, -2) - 20 * sh(a, -1) + 90 * a + 60 * sh(a, 1) - 5 * sh(a, 2)) / 128
            linm = lambda a: (3 * sh(a, 3) - 20 * sh(a, 2) + 90 * sh(a, 1) + 60 * a - 5 * sh(a, -1)) / 128
        else:
            lin = lambda a: (-sh(a, -1) + 6 * a + 3 * sh(a, 1)) / 8
            linm = lambda a: (-sh(a, 2) + 6 * sh(a, 1) + 3 * a) / 8
        qp, qm = lin(q), linm(q)          # Q+ and Q- at j + 1/2
        E = _euler_x_flux(q, mx, my)
        fp, fm = 0.5 * (E + A * q), 0.5 * (E - A * q)
        fpm = 0.5 * (_euler_x_flux(qp, mx, my) + A * qp)
        fmm = 0.5 * (_euler_x_flux(qm, mx, my) - A * qm)
        H = tab["hmid"][0] * (fpm + fmm) + tab["hmid"][1] * (sh(fpm, -1) + sh(fmm, 1))
        for k in range(-3, 4):
            H = H + tab["hnode"][k + 3] * (sh(fp, k) + sh(fm, 1 - k))
        total += H - sh(H, -1)
    return -total / (h * h)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_linear_weights_reduce_to_linear_upwind_operator(scheme):
    n, L = 16, 8.0
    x, y, per = I.periodic_square(n, L, 0.0, seed=0)
    q = I.isentropic_vortex(x, y, (4.0, 4.0), strength=3.0, free=(1.0, 0.5, 0.2, 1.0), period=(L, L))
    cfg = _cfg(scheme=scheme, period=per, linear_weights=1)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    want = _closed_form_linear_rhs(scheme, q, L / n)
    assert np.allclose(R, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("scheme,order,ns", [(0, 3, (128, 256)), (1, 3, (128, 256)), (2, 5, (128, 256)),
                                            (3, 5, (128, 256)), (4, 7, (128, 256))])
def test_design_order_on_curved_grid(scheme, order, ns):
    # a stationary isentropic vortex is an exact steady solution: the residual converges
    # at the design order (linear weights isolate the scheme's order)
    errs = []
    for n in ns:
        x, y, per = I.curved_periodic(n, 16.0, 0.1, origin=(-8.0, -8.0))
        cfg = _cfg(scheme=scheme, period=per, linear_weights=1)
        q = I.isentropic_vortex(x, y, (0.0, 0.0), free=(1.0, 0.0, 0.0, 1.0))
        R = O.rhs(cfg, O.metrics(cfg, x, y), q)
        errs.append(math.sqrt((R * R).mean()))
    assert math.log2(errs[0] / errs[1]) > order - 0.3


def test_line_lambda_closed_form():
    ni, nj, h, s = 10, 9, 0.5, 0.2
    x, y, per = _affine(ni, nj, h, s)
    cfg = _cfg(period=per)
    M = O.metrics(cfg, x, y)
    u, v, rho, p = 0.7, -0.4, 1.3, 0.9
    q = I.uniform_state(x.shape, rho, u, v, p)
    lx, le = O.line_lambda(cfg, M, q)
    c = math.sqrt(GAMMA * p / rho)
    # xi^ = (y_eta, -x_eta) = (h, -s); eta^ = (-y_xi, x_xi) = (0, h)
    assert np.allclose(lx, 1.1 * (abs(h * u - s * v) + c * math.hypot(h, s)), rtol=1e-14)
    assert np.allclose(le, 1.1 * (abs(h * v) + c * h), rtol=1e-14)
    dt = O.cfl_dt(cfg, M, q, 0.5)
    want = 0.5 / ((abs(h * u - s * v) + c * math.hypot(h, s) + abs(h * v) + c * h) / (h * h))
    assert dt == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (2, 2, 2, 2), (4, 4, 4, 4), (0, 0, 3, 3)])
def test_uniform_flow_kept_by_boundaries(bc):
    # uniform flow along x (parallel to the j-faces, so slip walls there keep it)
    x, y = I.paper_random_grid(21, 21, 4.0, 0.3, seed=9)
    if bc[0] == 0:
        n, L = 21, 4.0
        x, y, per = I.periodic_square(n, L, 0.0, seed=0)
        xr, yr = I.randomize(x, y, L / n, L / n, np.where((np.arange(n) >= 5) & (np.arange(n) < n - 5), 0.3, 0.0)[:, None] * np.ones((1, n)), seed=9)
        x, y = xr, yr
    else:
        per = ((0.0, 0.0), (0.0, 0.0))
    q0 = _uniform_q(0.6, 0.0, 1.0, 1.0 / GAMMA)
    st = np.tile(q0, (4, 1))
    cfg = _cfg(scheme=2, bc=bc, bc_state=st, period=per)
    R = O.rhs(cfg, O.metrics(cfg, x, y), I.uniform_state(x.shape, 1.0, 0.6, 0.0, 1.0 / GAMMA))
    assert np.abs(R).max() < 1e-11


# Boundary rules (readings: the paper treats no boundaries) pinned to what each rule means,
# on a uniform grid turned by 0.3 rad (so that both velocity components cross the i-faces),
# periodic in j, with a state that varies at the faces.
_TH = 0.3


def _turned_grid(i0, ni, nj, h=0.25):
    c, s = math.cos(_TH), math.sin(_TH)
    i, j = np.arange(i0, i0 + ni, dtype=np.float64), np.arange(nj, dtype=np.float64)
    X, Y = np.broadcast_to(h * i[None, :], (nj, ni)), np.broadcast_to(h * j[:, None], (nj, ni))
    return c * X - s * Y, s * X + c * Y, ((0.0, 0.0), (-s * h * nj, c * h * nj))


def _face_state(x, y):
    c, s = math.cos(_TH), math.sin(_TH)
    X, Y = c * x + s * y, -s * x + c * y
    rng = np.random.default_rng(4)
    rho = 1 + 0.2 * np.exp(-((X - 1.0) ** 2 + (Y - 2.0) ** 2)) + 0.02 * rng.standard_normal(X.shape)
    u = 0.3 + 0.2 * np.sin(Y) + 0.02 * rng.standard_normal(X.shape)
    v = -0.2 + 0.1 * np.cos(X)
    p = 1 + 0.1 * np.exp(-((X - 0.5) ** 2 + (Y - 1.0) ** 2))
    return I.conservative(rho, c * u - s * v, s * u + c * v, p)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_slip_wall_is_a_symmetry_plane(scheme):
    """Next to a slip wall the right-hand side is that of the doubled domain: the block and
    its mirror image about the wall line, velocity reflected (node 0 lies on the wall)."""
    n, nj = 14, 16
    x, y, per = _turned_grid(0, n, nj)
    q = _face_state(x, y)
    cfg = _cfg(scheme=scheme, bc=(3, 1, 0, 0), period=per)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    xd, yd, _ = _turned_grid(-(n - 1), 2 * n - 1, nj)
    qd = np.concatenate([q[:, :, :0:-1], q], axis=2)
    m = qd[:, :, :n - 1]
    c, s = math.cos(_TH), math.sin(_TH)
    un = m[1] * c + m[2] * s
    m[1] -= 2 * un * c
    m[2] -= 2 * un * s
    cfgd = _cfg(scheme=scheme, bc=(1, 1, 0, 0), period=per)
    Rd = O.rhs(cfgd, O.metrics(cfgd, xd, yd), qd)
    assert np.abs(Rd[:, :, n - 1:] - R).max() < 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_transmissive_face_is_a_constant_continuation(scheme):
    """A transmissive face gives the right-hand side of the block continued by copies of its
    boundary node (on a uniform grid the continued metrics equal the boundary node's, so the
    line maxima do not change either)."""
    n, nj, pad = 14, 16, 12
    x, y, per = _turned_grid(0, n, nj)
    q = _face_state(x, y)
    cfg = _cfg(scheme=scheme, bc=(1, 1, 0, 0), period=per)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    xp, yp, _ = _turned_grid(-pad, n + pad, nj)
    qp = np.concatenate([np.repeat(q[:, :, :1], pad, axis=2), q], axis=2)
    Rp = O.rhs(cfg, O.metrics(cfg, xp, yp), qp)
    assert np.abs(Rp[:, :, pad:] - R).max() < 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("scheme", [0, 2, 4])
def test_dirichlet_face_holds_its_own_state(scheme):
    """A Dirichlet face gives the right-hand side of the block continued by nodes that hold
    that face's prescribed state.  Each face has its own state, and each is slower than the
    interior's fastest wave, so the continued nodes leave the line maxima alone."""
    n, nj, pad = 14, 16, 12
    x, y, per = _turned_grid(0, n, nj)
    q = _face_state(x, y)
    st = np.stack([I.conservative(1.1, 0.05, 0.0, 0.9), I.conservative(0.9, -0.05, 0.02, 1.05),
                   I.conservative(1.0, 0.0, 0.0, 1.0), I.conservative(1.0, 0.0, 0.0, 1.0)])
    cfg = _cfg(scheme=scheme, bc=(2, 2, 0, 0), period=per, bc_state=st)
    R = O.rhs(cfg, O.metrics(cfg, x, y), q)
    xp, yp, _ = _turned_grid(0, n + pad, nj)
    qp = np.concatenate([q, np.repeat(st[1][:, None, None], nj, axis=1).repeat(pad, axis=2)], axis=2)
    cfgp = _cfg(scheme=scheme, bc=(2, 1, 0, 0), period=per, bc_state=st)
    Rp = O.rhs(cfgp, O.metrics(cfgp, xp, yp), qp)
    assert np.abs(Rp[:, :, :n] - R).max() < 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("scheme", [0, 2, 4])
def test_far_field_is_dirichlet_on_inflow_and_transmissive_on_outflow(scheme):
    x, y, per = _turned_grid(0, 14, 16)
    q = _face_state(x, y)
    c, s = math.cos(_TH), math.sin(_TH)
    for speed, same_as in ((0.5, 2), (-0.5, 1)):   # prescribed velocity into / out of the i- face
        st = np.tile(I.conservative(1.1, c * speed, s * speed, 0.9), (4, 1))
        out = []
        for bc0 in (4, same_as):
            cfg = _cfg(scheme=scheme, bc=(bc0, 1, 0, 0), period=per, bc_state=st)
            out.append(O.rhs(cfg, O.metrics(cfg, x, y), q))
        assert np.array_equal(out[0], out[1])


def test_rk3_third_order_in_time():
    n, L = 24, 8.0
    x, y, per = I.periodic_square(n, L, 0.0, seed=0)
    q0 = I.isentropic_vortex(x, y, (4.0, 4.0), strength=3.0, free=(1.0, 1.0, 0.5, 1.0), period=(L, L))
    cfg = _cfg(scheme=2, period=per)
    M = O.metrics(cfg, x, y)
    T = 0.4
    ref = O.rk3(cfg, M, q0, T / 64, 64)
    errs = [np.abs(O.rk3(cfg, M, q0, T / k, k) - ref).max() for k in (4, 8)]
    assert math.log2(errs[0] / errs[1]) > 2.7


def test_exact_riemann_solver_jump_conditions():
    g = 1.4
    WL, WR = np.array([1.0, 0.0, 1.0]), np.array([0.125, 0.0, 0.1])
    x = np.linspace(0.0, 1.0, 4001)
    W = O.riemann_exact(g, WL, WR, 0.5, 0.2, x)
    rho, u, p = W[:, 0], W[:, 1], W[:, 2]
    # star pressure and velocity are constant across the contact
    mid = (x > 0.55) & (x < 0.84)
    assert np.ptp(p[mid]) < 1e-12 and np.ptp(u[mid]) < 1e-12
    ps, us = p[mid][0], u[mid][0]
    # shock (right-moving into the right state): Rankine-Hugoniot for mass and momentum
    rs = rho[(x > 0.72) & (x < 0.84)][0]
    S = (rs * us - WR[0] * WR[1]) / (rs - WR[0])
    assert (rs * (us - S) ** 2 + ps) == pytest.approx(WR[0] * (WR[1] - S) ** 2 + WR[2], rel=1e-10)
    Es, ER = ps / (g - 1) + 0.5 * rs * us * us, WR[2] / (g - 1)
    assert (us * (Es + ps) - S * Es) == pytest.approx(WR[1] * (ER + WR[2]) - S * ER, rel=1e-10)
    # rarefaction: isentropic, and the left Riemann invariant u + 2c/(g-1) is constant
    fan = (x > 0.27) & (x < 0.48)
    assert np.allclose(p[fan] / rho[fan] ** g, WL[2] / WL[0] ** g, rtol=1e-12)
    c = np.sqrt(g * p[fan] / rho[fan])
    assert np.allclose(u[fan] + 2 * c / (g - 1), 2 * math.sqrt(g) / (g - 1), rtol=1e-12)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_sod_against_exact_solution(scheme):
    x, y, q, per = I.sod_1d(200)
    cfg = _cfg(scheme=scheme, period=per, bc=(1, 1, 0, 0))
    M = O.metrics(cfg, x, y)
    mass0 = q[0].sum()
    t = 0.0
    while t < 0.2 - 1e-14:
        dt = min(O.cfl_dt(cfg, M, q, 0.5), 0.2 - t)
        q = O.rk3(cfg, M, q, dt)
        t += dt
    ex = O.riemann_exact(GAMMA, [1, 0, 1], [0.125, 0, 0.1], 0.5, 0.2, x[0])
    assert np.abs(q[0, 0] - ex[:, 0]).mean() < 5e-3
    assert abs(q[0].sum() - mass0) < 1e-13 * mass0
