"""Pins of the oracle's three-dimensional path (Sections 2.1-2.2: five variables, the
symmetric conservative metrics of Eq. 2.4, the Jacobian of Eq. 2.5, three sweeps), CPU only.

* On a two-dimensional grid extruded along k with a state that does not depend on k, the
  flux differences of the three-dimensional right-hand side equal those of the (separately
  pinned) two-dimensional oracle and the w equation stays at round-off.  J^-1 itself differs:
  Eq. 2.5's zeta_z^ is a conservative difference of products, which equals the
  two-dimensional x_xi y_eta - x_eta y_xi only up to truncation.
* A uniform flow on a randomised three-dimensional grid keeps a round-off residual for every
  scheme (less in long double); with another scheme's operator in the metrics it does not.
* The eigenvectors diagonalise a Jacobian of the flux written here independently; with linear
  weights the right-hand side turns with the grid under a rotation; the right-hand side
  telescopes on periodic grids; a stationary vortex on a warped grid converges at the design
  order."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

GAMMA = 1.4
G = 4


def _extruded(scheme, nk=6):
    x, y, per = I.periodic_square(14, 8.0, 0.2, seed=21, nj=12)
    q2 = I.isentropic_vortex(x, y, (4.0, 4.0), strength=5.0, free=(1.0, 1.0, 0.5, 1.0), period=(8.0, 8.0))
    X, Y, Z = I.extrude(x, y, nk)
    per3 = ((8.0, 0.0, 0.0), (0.0, 8.0, 0.0), (0.0, 0.0, float(nk)))
    Q3 = np.stack([q2[0], q2[1], q2[2], 0.0 * q2[0], q2[3]])[:, None].repeat(nk, axis=1)
    return x, y, per, q2, X, Y, Z, per3, Q3


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_extruded_grid_reduces_to_two_dimensions(scheme):
    x, y, per, q2, X, Y, Z, per3, Q3 = _extruded(scheme)
    c2, c3 = dict(scheme=scheme, period=per), dict(scheme=scheme, period=per3, bc=(0,) * 6)
    M2, M3 = O.metrics(c2, x, y), O.metrics3(c3, X, Y, Z)
    # the direction metrics of xi and eta are the two-dimensional ones (dz = 1); their z parts
    # and zeta_x^, zeta_y^ vanish
    k = G + 2
    for p3, p2 in ((0, 0), (1, 1), (3, 2), (4, 3)):
        assert np.abs(M3[p3, k] - M2[p2]).max() < 1e-13
    for p3 in (2, 5, 6, 7):
        assert np.abs(M3[p3, k]).max() < 1e-13
    # flux differences R = -dQ/dt J^-1
    R3 = O.rhs3(c3, M3, Q3) * M3[9, G:-G, G:-G, G:-G][None]
    R2 = O.rhs(c2, M2, q2) * M2[4, G:-G, G:-G][None]
    scale = np.abs(R2).max()
    for v3, v2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
        assert np.abs(R3[v3] - R2[v2][None]).max() < 1e-13 * scale
    assert np.abs(R3[3]).max() < 1e-14 * scale


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_free_stream_on_randomised_cube(scheme):
    x, y, z, per = I.periodic_cube(12, 6.0, 0.2, seed=5)
    cfg = dict(scheme=scheme, period=per, bc=(0,) * 6)
    q0 = [1.0, 0.5, 0.3, -0.2, 2.5]
    r64 = O.fsp_residual3(cfg, x, y, z, q0)
    r80 = O.fsp_residual3(cfg, x, y, z, q0, wide=True)
    assert r64 < 1e-12 and r80 < 1e-3 * r64
    # negative control: metrics from another scheme's operator
    Mbad = O.metrics3(dict(cfg, scheme=(scheme + 2) % 5), x, y, z)
    Q = np.array(q0)[:, None, None, None] * np.ones((5,) + x.shape)
    assert np.abs(O.rhs3(cfg, Mbad, Q)).max() > 1e-5


def test_free_stream_with_transmissive_faces():
    """Uniform flow on a randomised non-periodic box (reflected ghost coordinates, copied ghost
    states) is kept for every scheme."""
    x, y, z, _ = I.periodic_cube(14, 6.0, 0.2, seed=8)
    for scheme in range(5):
        for bc in ((1,) * 6, (0, 0, 1, 1, 0, 0)):
            per = ((6.0, 0.0, 0.0), (0.0, 6.0, 0.0), (0.0, 0.0, 6.0))
            cfg = dict(scheme=scheme, period=per, bc=bc)
            assert O.fsp_residual3(cfg, x, y, z, [1.0, 0.5, 0.3, -0.2, 2.5]) < 1e-12, (scheme, bc)


def _flux_np(q, m):
    rho, u, v, w = q[0], q[1] / q[0], q[2] / q[0], q[3] / q[0]
    p = (GAMMA - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w))
    U = m[0] * u + m[1] * v + m[2] * w
    return np.array([rho * U, rho * u * U + m[0] * p, rho * v * U + m[1] * p, rho * w * U + m[2] * p,
                     (q[4] + p) * U])


@pytest.mark.parametrize("n", [(0.6, -0.48, 0.64), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, 0.6, -0.8),
                               (0.577, 0.577, 0.578)])
def test_eigenvectors(n):
    n = np.array(n) / np.linalg.norm(n)
    rng = np.random.default_rng(4)
    for _ in range(5):
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        u = rng.uniform(-1.5, 1.5, 3)
        q = I.conservative3(rho, *u, p)
        L, R = O.eig3(GAMMA, q, n)
        assert np.abs(L @ R - np.eye(5)).max() < 1e-13
        # Jacobian of the flux along n by central differences
        h = 1e-6
        A = np.zeros((5, 5))
        for c in range(5):
            dq = np.zeros(5)
            dq[c] = h * max(1.0, abs(q[c]))
            A[:, c] = (_flux_np(q + dq, n) - _flux_np(q - dq, n)) / (2 * dq[c])
        c_s = math.sqrt(GAMMA * p / rho)
        Un = u @ n
        lam = np.array([Un - c_s, Un, Un, Un, Un + c_s])
        assert np.abs(A @ R - R * lam[None]).max() < 1e-6
        # the tangents are unit vectors orthogonal to n and to each other
        t1, t2 = R[1:4, 2], R[1:4, 3]
        assert abs(t1 @ n) < 1e-14 and abs(t2 @ n) < 1e-14 and abs(t1 @ t2) < 1e-14
        assert abs(t1 @ t1 - 1) < 1e-14 and abs(t2 @ t2 - 1) < 1e-14


def _rotation(axis, angle):
    a = np.asarray(axis, dtype=float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


@pytest.mark.parametrize("scheme", [0, 3, 4])
def test_rotation_with_linear_weights(scheme):
    """With linear weights the characteristic projection and reconstruction compose to the
    identity on each stencil, so the tangent basis cannot matter: turning the grid, its periods
    and the velocity turns the momentum part of the right-hand side."""
    x, y, z, per = I.periodic_cube(10, 5.0, 0.2, seed=9)
    q = I.random_state3(x.shape, seed=3)
    Rot = _rotation((1.0, 2.0, 3.0), 0.5)
    P = np.stack([x, y, z])
    Pr = np.einsum("ab,b...->a...", Rot, P)
    perr = tuple(tuple(Rot @ np.array(per[a])) for a in range(3))
    qr = q.copy()
    qr[1:4] = np.einsum("ab,b...->a...", Rot, q[1:4])
    c = dict(scheme=scheme, linear_weights=1, period=per, bc=(0,) * 6)
    cr = dict(c, period=perr)
    R = O.rhs3(c, O.metrics3(c, x, y, z), q)
    Rr = O.rhs3(cr, O.metrics3(cr, *Pr), qr)
    scale = np.abs(R).max()
    assert np.abs(Rr[0] - R[0]).max() < 1e-11 * scale
    assert np.abs(Rr[4] - R[4]).max() < 1e-11 * scale
    assert np.abs(Rr[1:4] - np.einsum("ab,b...->a...", Rot, R[1:4])).max() < 1e-11 * scale


@pytest.mark.parametrize("scheme", [1, 2])
def test_conservation(scheme):
    x, y, z, per = I.periodic_cube(10, 5.0, 0.2, seed=10)
    q = I.random_state3(x.shape, seed=4)
    c = dict(scheme=scheme, period=per, bc=(0,) * 6)
    M = O.metrics3(c, x, y, z)
    R = O.rhs3(c, M, q) * M[9, G:-G, G:-G, G:-G][None]
    assert np.abs(R.sum(axis=(1, 2, 3))).max() < 1e-12 * np.abs(R).sum()


def _warped_cube(n, L=8.0, amp=0.15):
    """A smooth periodic warp of the cube: each coordinate moves by amp h sin of the others."""
    h = L / n
    k, j, i = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), np.arange(n, dtype=float),
                          indexing="ij")
    s = 2 * math.pi / n
    x = h * i + amp * h * np.sin(s * j) * np.sin(s * k) * n / 8
    y = h * j + amp * h * np.sin(s * k) * np.sin(s * i) * n / 8
    z = h * k + amp * h * np.sin(s * i) * np.sin(s * j) * n / 8
    return x, y, z, ((L, 0.0, 0.0), (0.0, L, 0.0), (0.0, 0.0, L))


@pytest.mark.parametrize("scheme,order", [(0, 2.5), (2, 4.0), (4, 5.3)])
def test_design_order_stationary_vortex(scheme, order):
    """A stationary isentropic vortex (axis along z, no free stream) is a steady solution, so
    the right-hand side is the truncation error; with linear weights on a smoothly warped grid
    (curved in all three directions) it falls at close to the design order between 32^3 and
    48^3 (measured 2.7, 4.3 and 5.7 for WENOIU3-1MP, WENOIU5-1MP and WENOIU7-1MP, still
    rising: the vortex core spans five nodes at 48^3).  The vortex is narrow (e^{1 - r^2}, core
    0.8) so that its periodic images meet below 1e-10."""
    err = []
    for n in (32, 48):
        x, y, z, per = _warped_cube(n)
        q2 = I.isentropic_vortex(x.reshape(-1, n), y.reshape(-1, n), (4.0, 4.0), strength=1.0,
                                 free=(1.0, 0.0, 0.0, 1.0), period=(8.0, 8.0), alpha=1.0,
                                 rc=0.8).reshape((4,) + x.shape)
        q = np.stack([q2[0], q2[1], q2[2], 0.0 * q2[0], q2[3]])
        c = dict(scheme=scheme, linear_weights=1, period=per, bc=(0,) * 6)
        R = O.rhs3(c, O.metrics3(c, x, y, z), q)
        err.append(math.sqrt(float((R * R).mean())))
    assert math.log(err[0] / err[1]) / math.log(1.5) > order, err


def test_operation_count_is_affine_in_the_line_length():
    """With linear weights each sweep's count per line is the same program for every line, so
    the count grows exactly affinely with the line length (the roofline's per-node figure is
    evaluated at the workload's size from two small grids)."""
    tot = []
    for n in (8, 10, 12):
        x, y, z, per = I.periodic_cube(n, 5.0, 0.2, seed=12, nj=6, nk=6)
        q = I.random_state3(x.shape, seed=2)
        c = dict(scheme=2, linear_weights=1, period=per, bc=(0,) * 6)
        tot.append(O.count_flops3(c, O.metrics3(c, x, y, z), q)["xi"])
    assert tot[2] - tot[1] == tot[1] - tot[0] > 0


@pytest.mark.parametrize("bc", [(0,) * 6, (1,) * 6])
def test_metrics_exact_on_affine_grids(bc):
    """On an affine grid x = A (i, j, k) + b every derivative in Eq. 2.4 is exact (the central
    operators are exact on linear data, and the odd reflection of the ghost coordinates keeps
    the grid affine), so the metrics are the cofactors of A (row d of the inverse times det A)
    and J^-1 = det A, at every node including the ghosts."""
    A = np.array([[0.9, 0.2, -0.1], [0.15, 1.1, 0.25], [-0.05, 0.3, 0.8]])
    n = 14
    k, j, i = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), np.arange(n, dtype=float),
                          indexing="ij")
    X = [A[c, 0] * i + A[c, 1] * j + A[c, 2] * k + 0.3 * c for c in range(3)]
    per = tuple(tuple(n * A[:, a]) for a in range(3))
    for scheme in range(5):
        M = O.metrics3(dict(scheme=scheme, period=per, bc=bc), *X)
        det = np.linalg.det(A)
        cof = det * np.linalg.inv(A)          # row d: the metric vector of direction d
        for d in range(3):
            for c in range(3):
                assert np.abs(M[3 * d + c] - cof[d, c]).max() < 1e-12, (scheme, d, c)
        assert np.abs(M[9] - det).max() < 1e-12
