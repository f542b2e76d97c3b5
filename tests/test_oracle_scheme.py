"""Pins of the oracle's scheme algebra against what the paper fixes (CPU only).

* the printed central operators (Eqs. 3.7, 3.9, 3.19, 3.21, and the Appendix's eighth-order
  one for WENOIU7-1MP) equal the central-scheme decomposition (Eq. 2.7) of the printed h+
  formulas (Eqs. 3.4, 3.8, 3.16, 3.20, Appendix scheme (1) with alpha = 1);
* every h+ formula and central operator has its design order on polynomials;
* the WENO interpolation of Table 1 is exact on polynomials with linear weights,
  non-oscillatory at a step, and the indicators equal the printed Eq. (3.22);
* the mappings (3.15)/(3.23) have the fixed points and flatness the paper states;
* the eigenvectors diagonalise the metric-weighted flux Jacobian.
"""
import math

import numpy as np
import pytest

import oracle as O

SCHEMES = [0, 1, 2, 3, 4]
ORDER = {0: 3, 1: 3, 2: 5, 3: 5, 4: 7}


def _csd(tab):
    """Node and midpoint coefficients of (H_{j+1/2} - H_{j-1/2}) with H = (h+ + h-)/2."""
    hn = {k: tab["hnode"][k + 3] for k in range(-3, 4)}
    hm = {0: tab["hmid"][0], -1: tab["hmid"][1]}
    cH = {}
    for k, c in hn.items():               # h+ node offsets k, h- mirrored to 1 - k
        cH[k] = cH.get(k, 0.0) + 0.5 * c
        cH[1 - k] = cH.get(1 - k, 0.0) + 0.5 * c
    cM = {}
    for m, c in hm.items():               # h+ midpoint offsets m, h- mirrored to -m
        cM[m] = cM.get(m, 0.0) + 0.5 * c
        cM[-m] = cM.get(-m, 0.0) + 0.5 * c
    node = {o: cH.get(o, 0.0) - cH.get(o + 1, 0.0) for o in range(-5, 6)}
    mid = {o: cM.get(o, 0.0) - cM.get(o + 1, 0.0) for o in range(-5, 6)}
    return node, mid


@pytest.mark.parametrize("scheme", SCHEMES)
def test_printed_central_operator_is_csd_of_printed_h(scheme):
    tab = O.scheme_table(scheme)
    node, mid = _csd(tab)
    for k in (1, 2, 3, 4):
        a = tab["cnode"][k - 1]
        assert node[k] == pytest.approx(a, abs=1e-15)
        assert node[-k] == pytest.approx(-a, abs=1e-15)
    assert node[0] == pytest.approx(0.0, abs=1e-15)
    assert node[5] == pytest.approx(0.0, abs=1e-15) and node[-5] == pytest.approx(0.0, abs=1e-15)
    # midpoint j+1/2+m' <-> offset m'; b_{1/2} on (f~_{j+1/2} - f~_{j-1/2}), b_{3/2} likewise
    b12, b32 = tab["cmid"]
    assert mid[0] == pytest.approx(b12, abs=1e-15) and mid[-1] == pytest.approx(-b12, abs=1e-15)
    assert mid[1] == pytest.approx(b32, abs=1e-15) and mid[-2] == pytest.approx(-b32, abs=1e-15)
    for o in (-4, -3, 2, 3, 4):
        assert mid[o] == pytest.approx(0.0, abs=1e-15)


def _h_plus(tab, f, j):
    """h+_{j+1/2} on unit spacing with exact midpoint values f(j + 1/2 + m)."""
    h = sum(tab["hmid"][-m] * f(j + 0.5 + m) for m in (0, -1))
    return h + sum(tab["hnode"][k + 3] * f(j + k) for k in range(-3, 4))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_h_formula_design_order(scheme):
    tab = O.scheme_table(scheme)
    p = ORDER[scheme]
    j = 0.3  # any base point
    for d in range(0, p + 2):
        f = lambda x, d=d: x ** d
        fp = d * j ** (d - 1) if d > 0 else 0.0
        got = _h_plus(tab, f, j) - _h_plus(tab, f, j - 1)
        if d <= p:
            assert got == pytest.approx(fp, abs=1e-12), (d, got, fp)
        else:  # the leading error term of the accuracy relation is nonzero
            assert abs(got - fp) > 1e-6


@pytest.mark.parametrize("scheme", SCHEMES)
def test_central_operator_order(scheme):
    tab = O.scheme_table(scheme)
    q = ORDER[scheme] + 1  # 4, 6 or 8
    j = -0.2
    for d in range(0, q + 2):
        f = lambda x, d=d: x ** d
        got = sum(tab["cnode"][k - 1] * (f(j + k) - f(j - k)) for k in (1, 2, 3, 4))
        got += tab["cmid"][0] * (f(j + 0.5) - f(j - 0.5)) + tab["cmid"][1] * (f(j + 1.5) - f(j - 1.5))
        want = d * j ** (d - 1) if d > 0 else 0.0
        if d <= q:
            assert got == pytest.approx(want, abs=1e-12)
        elif d == q + 1:
            assert abs(got - want) > 1e-6


@pytest.mark.parametrize("r,deg", [(2, 2), (3, 4)])
def test_linear_weno_exact_on_polynomials(r, deg):
    rng = np.random.default_rng(1)
    for d in range(deg + 1):
        c = rng.normal(size=d + 1)
        poly = lambda x: sum(c[k] * x ** k for k in range(d + 1))
        u = np.array([poly(m) for m in range(-2, 3)])
        assert O.weno(r, u, linw=1) == pytest.approx(poly(0.5), abs=1e-13)
    # one degree more is no longer exact
    u = np.array([float(m) ** (deg + 1) for m in range(-2, 3)])
    assert abs(O.weno(r, u, linw=1) - 0.5 ** (deg + 1)) > 1e-4


@pytest.mark.parametrize("r", [2, 3])
@pytest.mark.parametrize("ppm", [0, 1])
def test_weno_constant_and_step(r, ppm):
    eps = 1e-40 if ppm else 1e-6
    assert O.weno(r, np.full(5, 2.5), ppm=ppm, eps=eps) == pytest.approx(2.5, rel=1e-15)
    # a step between u_j and u_{j+1}: the interpolant stays on the smooth (left) side
    step = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    assert abs(O.weno(r, step, ppm=ppm, eps=eps)) < (1e-10 if ppm else 1e-2)
    # a step between u_{j-1} and u_j: for r = 3 the stencil {j, j+1, j+2} is chosen; for
    # r = 2 both three-point indicators of Section 5.1 see the step, so only a bounded
    # overshoot is required
    step2 = np.array([0.0, 0.0, 1.0, 1.0, 1.0])
    v = O.weno(r, step2, ppm=ppm, eps=eps)
    if r == 3:
        assert v == pytest.approx(1.0, abs=1e-10 if ppm else 1e-2)
    else:
        assert abs(v - 1.0) < 0.1


def test_smoothness_indicators_equal_printed_quadratic_forms():
    rng = np.random.default_rng(2)
    for _ in range(50):
        u = rng.normal(size=5)
        a, b, c, d, e = u  # u_{j-2} .. u_{j+2}
        printed = np.array([
            (4 * a * a - 19 * a * b + 25 * b * b + 11 * a * c - 31 * b * c + 10 * c * c) / 3,
            (4 * b * b - 13 * b * c + 13 * c * c + 5 * b * d - 13 * c * d + 4 * d * d) / 3,
            (10 * c * c - 31 * c * d + 25 * d * d + 11 * c * e - 19 * d * e + 4 * e * e) / 3,
        ])  # Eq. (3.22)
        assert np.allclose(O.smoothness(u), printed, rtol=1e-12, atol=1e-13)
    assert np.all(O.smoothness(np.full(5, 3.7)) == 0.0)


@pytest.mark.parametrize("order,Cs", [(2, (0.25, 0.75)), (3, (1 / 16, 10 / 16, 5 / 16))])
def test_ppm_mapping_properties(order, Cs):
    for C in Cs:
        assert O.ppm(order, 0.0, C) == pytest.approx(0.0, abs=1e-15)
        assert O.ppm(order, 1.0, C) == pytest.approx(1.0, abs=1e-14)
        assert O.ppm(order, C, C) == pytest.approx(C, abs=1e-15)
        h = 1e-4
        d1 = (O.ppm(order, C + h, C) - O.ppm(order, C - h, C)) / (2 * h)
        assert abs(d1) < 5 * h  # g'(C) = 0
        if order == 3:           # g''(C) = 0 too: the change is O(h^3)
            assert abs(O.ppm(order, C + h, C) - C) < 1e-10
        ws = np.linspace(0, 1, 201)
        g = np.array([O.ppm(order, w, C) for w in ws])
        assert np.all(np.diff(g) >= -1e-15)


def _flux(q, mx, my, gamma=1.4):
    rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
    p = (gamma - 1) * (q[3] - 0.5 * rho * (u * u + v * v))
    U = mx * u + my * v
    return np.array([rho * U, rho * u * U + mx * p, rho * v * U + my * p, (q[3] + p) * U])


def test_eigenvectors_diagonalise_flux_jacobian():
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho, u, v, p = rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.5, 2)
        q = np.array([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])
        m = rng.normal(size=2)
        n = m / np.linalg.norm(m)
        L, R = O.eig(1.4, q, n[0], n[1])
        assert np.allclose(L @ R, np.eye(4), atol=1e-13)
        # Jacobian of the metric-weighted flux by the complex step (exact to round-off)
        A = np.empty((4, 4))
        for k in range(4):
            dq = np.zeros(4, dtype=complex)
            dq[k] = 1e-30j
            A[:, k] = _flux(q + dq, m[0], m[1]).imag / 1e-30
        c = math.sqrt(1.4 * p / rho)
        U = m[0] * u + m[1] * v
        lam = np.diag([U - c * np.linalg.norm(m), U, U, U + c * np.linalg.norm(m)])
        assert np.allclose(L @ A @ R, lam, atol=1e-12 * (1 + np.abs(lam).max()))
