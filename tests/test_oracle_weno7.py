"""Pins of the oracle's seventh-order pieces (WENOIU7-1MP, the paper's Appendix) on the CPU.

* Table A1: each r = 4 candidate interpolates cubics exactly at x_{j+1/2}, and with the
  linear weights C^4_k the combination is the seven-point interpolant (exact to degree 6);
* smoothness indicators for r = 4 (a reading: the paper prints none): the definition that
  reproduces Eq. (3.22) for r = 3 -- the integral over [x_{j-1/2}, x_{j+1/2}] of the squared
  derivatives of the candidate's interpolating polynomial, scaled by powers of h -- derived
  here symbolically and compared with the oracle on random data;
* the fourth-order mapping of the Appendix: fixed points 0, C_k, 1, flat to third order at
  C_k, monotone;
* linear advection (Section 5.1 setup) converges at seventh order with RK4 steps
  dt ~ dx^(7/4), so the time error stays below the spatial one.
"""
import math

import numpy as np
import pytest

import oracle as O

C4 = (1 / 64, 21 / 64, 35 / 64, 7 / 64)


def test_table_a1_candidates_and_linear_weights():
    rng = np.random.default_rng(5)
    for d in range(7):
        c = rng.normal(size=d + 1)
        poly = lambda x: sum(c[k] * x ** k for k in range(d + 1))
        u = np.array([poly(m) for m in range(-3, 4)])
        assert O.weno(4, u, linw=1) == pytest.approx(poly(0.5), abs=1e-12)
    u = np.array([float(m) ** 7 for m in range(-3, 4)])
    assert abs(O.weno(4, u, linw=1) - 0.5 ** 7) > 1e-4
    # on a cubic every candidate is exact, so the nonlinear weights cannot matter
    c = rng.normal(size=4)
    cubic = lambda x: c[0] + c[1] * x + c[2] * x * x + c[3] * x ** 3
    u = np.array([cubic(m) for m in range(-3, 4)])
    for ppm in (0, 1):
        assert O.weno(4, u, ppm=ppm, eps=1e-6 if ppm == 0 else 1e-40) == pytest.approx(cubic(0.5), abs=1e-11)


def _indicators(r):
    """Indicators of the r candidates of u_{j-r+1+k .. j+k} by the definition, as functions
    of the seven values u_{j-3..j+3}."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    u = sp.symbols("u0:7")                    # u[m + 3] = u_{j+m}
    out = []
    for k in range(r):
        offs = list(range(-r + 1 + k, 1 + k))
        P = sp.interpolate([(o, u[o + 3]) for o in offs], x)
        half = sp.Rational(1, 2)
        out.append(sp.expand(sum(sp.integrate(sp.diff(P, x, l) ** 2, (x, -half, half)) for l in range(1, r))))
    return sp, u, out


def test_r3_definition_reproduces_printed_indicators():
    sp, u, IS = _indicators(3)
    a, b, c, d, e = u[1:6]                    # u_{j-2} .. u_{j+2}
    printed = [
        (4 * a * a - 19 * a * b + 25 * b * b + 11 * a * c - 31 * b * c + 10 * c * c) / sp.Integer(3),
        (4 * b * b - 13 * b * c + 13 * c * c + 5 * b * d - 13 * c * d + 4 * d * d) / sp.Integer(3),
        (10 * c * c - 31 * c * d + 25 * d * d + 11 * c * e - 19 * d * e + 4 * e * e) / sp.Integer(3),
    ]  # Eq. (3.22)
    for got, want in zip(IS, printed):
        assert sp.simplify(got - sp.expand(want)) == 0


def test_r4_indicators_follow_the_definition():
    sp, u, IS = _indicators(4)
    f = sp.lambdify(u, IS)
    rng = np.random.default_rng(6)
    for _ in range(30):
        v = rng.normal(size=7) * rng.uniform(0.1, 10)
        assert np.allclose(O.smoothness4(v), np.array(f(*v), dtype=float), rtol=1e-12, atol=1e-14)
    assert np.all(O.smoothness4(np.full(7, -2.3)) == 0.0)      # exactly zero on constants


def test_weno7_constant_and_step():
    assert O.weno(4, np.full(7, 1.75)) == pytest.approx(1.75, rel=1e-15)
    # a step between u_j and u_{j+1}: only candidate 0 is smooth, the interpolant stays left
    step = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    assert abs(O.weno(4, step)) < 1e-10
    # a step between u_{j-1} and u_j: candidate 3 (j .. j+3) is smooth
    step2 = np.array([0.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    assert O.weno(4, step2) == pytest.approx(1.0, abs=1e-10)


@pytest.mark.parametrize("C", C4)
def test_fourth_order_mapping(C):
    assert O.ppm(4, 0.0, C) == pytest.approx(0.0, abs=1e-15)
    assert O.ppm(4, 1.0, C) == pytest.approx(1.0, abs=1e-14)
    assert O.ppm(4, C, C) == pytest.approx(C, abs=1e-15)
    # g - C = -(w - C)^4 / C^3 below C and -(w - C)^4 / (C - 1)^3 above: the first three
    # derivatives vanish at C, so halving the distance divides the change by 16
    for s, K in ((-1, 1 / C ** 3), (1, -1 / (C - 1) ** 3)):
        for h in (1e-2, 5e-3):
            assert O.ppm(4, C + s * h, C) - C == pytest.approx(-s ** 4 * K * h ** 4 if s < 0 else K * h ** 4,
                                                                rel=1e-6)
    ws = np.linspace(0, 1, 401)
    g = np.array([O.ppm(4, w, C) for w in ws])
    assert np.all(np.diff(g) >= -1e-15)


def test_seventh_order_advection():
    errs = [O.advect1d_dt(4, n, 1.75)[0] for n in (40, 80, 160)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 6.8, orders
    assert errs[-1] < 5e-10
