"""Pins of the oracle's options beyond the paper's tested schemes (Section 7 names them as
further directions; the free parameter is Eqs. 3.5, 3.17 and the Appendix's scheme (1)):
the free-parameter one-midpoint forms, WENO-Z weights, and Steger-Warming / Van Leer
splitting of the midpoint flux.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

GAMMA = 1.4


# ---- free parameter of the one-midpoint forms ----------------------------------------------
def _h_on_monomial(tab, m):
    """h+_{j+1/2} of the scheme applied to f(x) = x^m with x_{j+1/2} = 0 and unit spacing: the
    node values f_{j+k} = (k - 1/2)^m and the exact midpoint value 0^m."""
    h = tab["hmid"][0] * (1.0 if m == 0 else 0.0)
    for k in range(-3, 4):
        h += tab["hnode"][k + 3] * (k - 0.5) ** m
    return h


@pytest.mark.parametrize("scheme", [0, 2, 4])
def test_alpha_one_is_the_printed_scheme(scheme):
    """The general forms at alpha = 1, and the central operator computed from them, equal the
    printed schemes (Eqs. 3.4/3.7, 3.16/3.19, the Appendix)."""
    printed = O.scheme_table(scheme)
    # alpha = 1 is taken from the printed table itself; approach it from both sides
    for a in (1.0 - 1e-9, 1.0 + 1e-9):
        t = O.scheme_table(scheme, a)
        for key in ("hmid", "hnode", "cnode", "cmid"):
            assert np.allclose(t[key], printed[key], rtol=0, atol=1e-8), key


@pytest.mark.parametrize("alpha", [0.7, 1.3])
def test_alpha_accuracy_relations(alpha):
    """h applied to monomials reproduces the printed accuracy relations: WENOIU5-1MP
    f - f''/24 + 7/5760 f'''' + (45 alpha - 64)/3840 f^(5) - (675 alpha - 983)/138240 f^(6)
    (after Eq. 3.17); WENOIU3-1MP f - f''/24 - (alpha/16 - 1/12) f''' + (3 alpha/128 - 37/1152)
    f'''' (after Eq. 3.5, whose f''' term is printed with the opposite sign: at alpha = 1 the
    printed h+ of Eq. 3.4 gives +1/48, the dissipative sign of an upwind-biased scheme); all at
    x_{j+1/2} = 0, dx = 1."""
    t3 = O.scheme_table(0, alpha)
    want3 = {0: 1.0, 1: 0.0, 2: -2.0 / 24, 3: -(alpha / 16 - 1.0 / 12) * 6, 4: (3 * alpha / 128 - 37.0 / 1152) * 24}
    for m, w in want3.items():
        assert _h_on_monomial(t3, m) == pytest.approx(w, abs=1e-13), (3, m)
    t5 = O.scheme_table(2, alpha)
    want5 = {0: 1.0, 1: 0.0, 2: -2.0 / 24, 3: 0.0, 4: 7.0 / 5760 * 24,
             5: (45 * alpha - 64) / 3840 * 120, 6: -(675 * alpha - 983) / 138240 * 720}
    for m, w in want5.items():
        assert _h_on_monomial(t5, m) == pytest.approx(w, abs=1e-12), (5, m)
    # WENOIU7-1MP: exact to the seventh order for any alpha (f^ of Eq. 3.3 has only even terms)
    t7 = O.scheme_table(4, alpha)
    fhat = {0: 1.0, 2: -2.0 / 24, 4: 7.0 / 5760 * 24, 6: -31.0 / 967680 * 720}
    for m in range(7):
        assert _h_on_monomial(t7, m) == pytest.approx(fhat.get(m, 0.0), abs=1e-12), (7, m)


@pytest.mark.parametrize("scheme", [0, 2, 4])
def test_alpha_central_operator_is_exact_and_preserves_free_stream(scheme):
    """With the alpha scheme's own central operator in the metrics the free stream is
    preserved on the randomised grid.  With the order-matched Lagrange midpoint interpolation
    that operator does not depend on alpha (the alpha-weighted midpoint difference and the node
    terms cancel exactly), so the check of the operator's alpha-dependence takes the two-point
    interpolation, where the alpha = 1 metrics with the alpha scheme (a mismatch) break the
    free stream."""
    x, y, per = I.periodic_square(24, 8.0, 0.2, seed=21)
    q = I.uniform_state(x.shape, 1.0, 0.5, 0.3, 1.0 / GAMMA)
    cfg = dict(scheme=scheme, period=per, scheme_alpha=1.3)
    M = O.metrics(cfg, x, y)
    assert np.abs(O.rhs(cfg, M, q)).max() < 1e-12
    M1 = O.metrics(dict(cfg, scheme_alpha=1.0), x, y)
    assert np.abs(M1 - M).max() < 1e-13 * np.abs(M).max()
    ca = dict(cfg, interp=1)
    Ma = O.metrics(ca, x, y)
    assert np.abs(O.rhs(ca, Ma, q)).max() < 1e-12
    assert np.abs(O.rhs(ca, O.metrics(dict(ca, scheme_alpha=1.0), x, y), q)).max() > 1e-6
    # a smooth state's right-hand side moves with alpha (the parameter is used)
    qv = I.isentropic_vortex(x, y, (4.0, 4.0), strength=3.0, free=(1.0, 0.5, 0.3, 1.0), period=(8.0, 8.0))
    assert np.abs(O.rhs(cfg, M, qv) - O.rhs(dict(cfg, scheme_alpha=1.0), M1, qv)).max() > 1e-6


def test_alpha_refused_for_two_midpoint_schemes():
    with pytest.raises(ValueError):
        O.metrics(dict(scheme=3, scheme_alpha=1.2, period=((1.0, 0.0), (0.0, 1.0))), np.zeros((12, 12)),
                  np.zeros((12, 12)))


# ---- WENO-Z weights --------------------------------------------------------------------------
@pytest.mark.parametrize("r", [2, 3, 4])
def test_weno_z_linear_weights_on_equal_indicators(r):
    """Where every indicator is the same (linear data), tau = 0 and the weights are the linear
    ones, so the interpolant is the linear one (exact on linear data)."""
    u = np.array([-3.0, -2.0, -1.0, 0.0, 1.0, 2.0, 3.0]) * 0.7 + 0.2
    z = O.weno_z(r, 1e-40, u)
    assert z == pytest.approx(0.2 + 0.35, abs=1e-14)


@pytest.mark.parametrize("r", [2, 3])
def test_weno_z_step_is_non_oscillatory(r):
    """Across a step the weights of the candidates that straddle it vanish: the midpoint value
    stays within the data's range."""
    u = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    z = O.weno_z(r, 1e-40, u)
    assert -1e-12 <= z <= 1.0 + 1e-12
    u2 = np.array([0.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    assert O.weno_z(r, 1e-40, u2) == pytest.approx(1.0, abs=1e-6)


@pytest.mark.parametrize("scheme,order", [(0, 3), (2, 5)])
def test_weno_z_design_order(scheme, order):
    """Scalar advection with WENO-Z weights (the setup of Table 3) converges at the design
    order."""
    errs = [O.advect1d_opts(scheme, n, 2.0, 1.25 if order < 7 else 1.75, 1)[0] for n in (40, 80)]
    assert math.log2(errs[0] / errs[1]) > order - 0.3


# ---- Steger-Warming and Van Leer at the midpoint ---------------------------------------------
def _random_states(n=200, seed=3):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.3, 2.0, n)
    u, v = rng.uniform(-3.0, 3.0, n), rng.uniform(-3.0, 3.0, n)
    p = rng.uniform(0.2, 2.0, n)
    mx, my = rng.uniform(-2.0, 2.0, n), rng.uniform(-2.0, 2.0, n)
    return rho, u, v, p, mx, my


@pytest.mark.parametrize("mode", [1, 2])
def test_midpoint_splittings_are_consistent(mode):
    """F+ + F- = E^ to rounding for random states and directions (subsonic and supersonic)."""
    for rho, u, v, p, mx, my in zip(*_random_states()):
        q = I.conservative(rho, u, v, p)
        fp, fm, e = O.split_flux(mode, q, mx, my, GAMMA)
        assert np.allclose(fp + fm, e, rtol=1e-13, atol=1e-13 * np.abs(e).max())


def test_midpoint_splittings_upwind_limits():
    """Supersonic along k: F+ = E^ and F- = 0 (Steger-Warming: all eigenvalues positive; Van
    Leer: M >= 1), and the reverse against k.  Van Leer's subsonic F+ meets E^ at M = 1."""
    q = I.conservative(1.0, 3.0, 0.5, 1.0)           # |u.n| > c along (1, 0.1)
    for mode in (1, 2):
        fp, fm, e = O.split_flux(mode, q, 1.0, 0.1, GAMMA)
        assert np.allclose(fp, e, rtol=1e-14) and np.allclose(fm, 0.0, atol=1e-14)
        fp, fm, e = O.split_flux(mode, q, -1.0, -0.1, GAMMA)
        assert np.allclose(fm, e, rtol=1e-14) and np.allclose(fp, 0.0, atol=1e-14)
    c = math.sqrt(GAMMA)                             # rho = p = 1
    for s in (1.0 - 1e-9, 1.0 + 1e-9):
        q = I.conservative(1.0, s * c, 0.0, 1.0)
        fp, fm, e = O.split_flux(2, q, 1.0, 0.0, GAMMA)
        assert np.allclose(fp, e, rtol=1e-7)


@pytest.mark.parametrize("mode", [1, 2])
def test_midpoint_splittings_keep_free_stream_and_conservation(mode):
    x, y, per = I.periodic_square(24, 8.0, 0.2, seed=21)
    cfg = dict(scheme=2, period=per, mid_split=mode)
    M = O.metrics(cfg, x, y)
    q = I.uniform_state(x.shape, 1.0, 0.5, 0.3, 1.0 / GAMMA)
    assert np.abs(O.rhs(cfg, M, q)).max() < 1e-12
    qr = I.random_state(x.shape, seed=9)
    R = O.rhs(cfg, M, qr)
    tot = (R * M[4, 4:-4, 4:-4][None]).sum(axis=(1, 2))
    assert np.abs(tot).max() < 1e-11 * np.abs(R * M[4, 4:-4, 4:-4][None]).sum()


@pytest.mark.parametrize("mode", [1, 2])
def test_midpoint_splittings_sod(mode):
    x, y, q, per = I.sod_1d(200)
    cfg = dict(scheme=2, period=per, bc=(1, 1, 0, 0), mid_split=mode)
    M = O.metrics(cfg, x, y)
    t = 0.0
    while t < 0.2 - 1e-14:
        dt = min(O.cfl_dt(cfg, M, q, 0.5), 0.2 - t)
        q = O.rk3(cfg, M, q, dt)
        t += dt
    ex = O.riemann_exact(GAMMA, [1, 0, 1], [0.125, 0, 0.1], 0.5, 0.2, x[0])
    assert np.abs(q[0, 0] - ex[:, 0]).mean() < 5e-3


@pytest.mark.parametrize("r,order", [(3, 9), (2, 7)])
def test_weno_z_weights_approach_the_linear_ones(r, order):
    """The global indicator is what makes WENO-Z: tau = |IS_0 - IS_2| is O(h^5) on smooth data
    while each IS is O(h^2), so the weights approach the linear ones fast and the interpolant
    differs from the linear one by far less than the interpolation error: on sin(x) the
    difference falls like h^10.5 (r = 3) and h^7.9 (r = 2).  A tau taken from neighbouring
    indicators for r = 3 would leave about h^6."""
    d = []
    for h in (0.4, 0.2):
        u = np.sin(0.3 + h * np.arange(-3, 4))
        d.append(abs(O.weno_z(r, 1e-40, u) - O.weno(r, u, ppm=0, linw=1)))
    assert math.log2(d[0] / d[1]) > order, d
