"""Pins of the oracle's four-midpoint seventh-order scheme (WENOIU7-4MP, the Appendix's scheme
(3), scheme index 5), CPU only.

* The printed delta^{c,(1)} is the central part (delta+ + delta-)/2 of the printed h+ (Eq. 2.7):
  recomputed here from the h+ coefficients, node terms and the midpoint terms to 5/2.
* h+ reproduces the flux f^ of Eq. (3.3) (f - f''/24 + 7/5760 f'''' - 31/967680 f^(6)) on
  monomials through degree 6 and not at degree 7: seventh order.
* Scalar advection (the Table 3 setup, RK4 with dt ~ dx^(7/4)) converges at seventh order.
* A uniform flow on a randomised periodic grid keeps a round-off residual (and not with the
  one-midpoint scheme's operator in the metrics); the right-hand side telescopes.
* The scheme reaches six nodes beyond a face: the oracle refuses non-periodic faces and linked
  blocks for it."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

S74 = 5


def _mids(t):
    # h+ coefficient of f+_{j+1/2+m}
    return {0: t["hmid"][0], -1: t["hmid"][1], -2: t["hmidx"][0], 1: t["hmidx"][1]}


def test_printed_central_operator_is_the_central_part_of_h():
    t = O.scheme_table(S74)
    n = lambda k: t["hnode"][k + 3] if -3 <= k <= 3 else 0.0
    a = [0.5 * (n(d) - n(d + 1) + n(1 - d) - n(-d)) for d in range(1, 5)]
    assert np.allclose(a, t["cnode"], atol=1e-15)
    c = _mids(t)
    cm = lambda m: c.get(m, 0.0)
    e = lambda p: cm(p) - cm(p + 1)            # delta+ coefficient of f~_{j+1/2+p}
    b = [0.5 * (e(p) - e(-p - 1)) for p in range(3)]   # b_{1/2}, b_{3/2}, b_{5/2}
    assert np.allclose(b, [t["cmid"][0], t["cmid"][1], t["cmid3"]], atol=1e-15)
    # as printed: a = (-32, 3) / 140, b = (1218, -17, -3) / 840
    assert np.allclose(t["cnode"][:2], [-32 / 140, 3 / 140]) and np.allclose(b, [1218 / 840, -17 / 840, -3 / 840])


def test_h_reproduces_the_flux_through_degree_six():
    t = O.scheme_table(S74)
    fhat = {0: 1.0, 2: -2.0 / 24, 4: 7.0 / 5760 * 24, 6: -31.0 / 967680 * 720}
    for deg in range(8):
        h = sum(cm * (float(m) ** deg if deg else 1.0) for m, cm in _mids(t).items())
        h += sum(t["hnode"][k + 3] * (k - 0.5) ** deg for k in range(-3, 4))
        if deg <= 6:
            assert h == pytest.approx(fhat.get(deg, 0.0), abs=1e-12), deg
        else:
            assert abs(h) > 1e-3


def test_seventh_order_advection():
    e = [O.advect1d_opts(S74, n, 2.0, 1.75, 0)[0] for n in (40, 80)]
    assert math.log2(e[0] / e[1]) > 6.5, e


def test_free_stream_and_conservation():
    x, y, per = I.periodic_square(24, 8.0, 0.2, seed=21)
    cfg = dict(scheme=S74, period=per)
    assert O.fsp_residual(cfg, x, y, [1.0, 0.5, 0.3, 2.5]) < 1e-12
    M = O.metrics(cfg, x, y)
    q0 = I.uniform_state(x.shape, 1.0, 0.5, 0.3, 1.0 / 1.4)
    assert np.abs(O.rhs(cfg, O.metrics(dict(cfg, scheme=4), x, y), q0)).max() > 1e-6
    q = I.random_state(x.shape, seed=9)
    R = O.rhs(cfg, M, q) * M[4, 4:-4, 4:-4][None]
    assert np.abs(R.sum(axis=(1, 2))).max() < 1e-12 * np.abs(R).sum()


def test_design_order_on_a_curved_grid():
    """A stationary vortex on a smoothly curved periodic grid with linear weights: the
    right-hand side is the truncation error and falls at about the seventh order (6.7 between
    64^2 and 128^2, as WENOIU7-1MP's 6.7; 6.0 between 32^2 and 64^2)."""
    err = []
    for n in (64, 128):
        x, y, per = I.curved_periodic(n, 8.0, warp=0.1)
        q = I.isentropic_vortex(x, y, (4.0, 4.0), strength=1.0, free=(1.0, 0.0, 0.0, 1.0), period=(8.0, 8.0),
                                alpha=1.0, rc=0.8)
        cfg = dict(scheme=S74, period=per, linear_weights=1)
        R = O.rhs(cfg, O.metrics(cfg, x, y), q)
        err.append(math.sqrt(float((R * R).mean())))
    assert math.log2(err[0] / err[1]) > 6.4, err


def test_non_periodic_faces_are_refused():
    x, y = I.riemann_grid(24, 0.2, 4)
    with pytest.raises(ValueError):
        O.metrics(dict(scheme=S74, bc=(1, 1, 1, 1)), x, y)
