"""Pins of the operation counter behind the roofline's algorithmic flops (CPU).

The counter runs the oracle with a scalar type that counts each + - * / and square root once.
* The final division by J^-1 (Eq. 2.2) is one operation per conserved variable and node.
* The line maxima: |U^| + c|k^| written out costs 22 operations per node, and alpha times the
  maximum one more per line.  The 22 are: u and v (2 divisions), the pressure
  (gamma - 1)(E - rho (u^2 + v^2)/2) (8), c = sqrt(gamma p / rho) (3), |mx u + my v| (3),
  c sqrt(mx^2 + my^2) (5) and the sum (1).
* With linear weights nothing depends on the data, so a sweep's count is exactly affine in
  the line length.
* The stored per-node counts are what the committed script computes now.
"""
import importlib
import json
import os

import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

CF = importlib.import_module("oracle.count_flops")   # the script (the package re-exports a function of that name)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _parts(scheme, ni, nj, **kw):
    x, y, per = I.periodic_square(ni, 6.0, 0.2, seed=11, nj=nj)
    q = I.isentropic_vortex(x, y, (3.1, 2.9), strength=3.0, free=(1.0, 0.5, 0.2, 1.0), period=(6.0, 6.0))
    cfg = dict(scheme=scheme, period=per, **kw)
    return O.count_flops_parts(cfg, O.metrics(cfg, x, y), q)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_closed_forms(scheme):
    ni, nj = 20, 14
    lx, sx, le, se, fin = _parts(scheme, ni, nj)
    assert fin == 4 * ni * nj
    assert lx == nj * (22 * ni + 1)
    assert le == ni * (22 * nj + 1)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_sweep_count_affine_in_line_length(scheme):
    nj = 12
    xi = [_parts(scheme, n, nj, linear_weights=1)[1] for n in (16, 24, 32)]
    assert xi[2] - xi[1] == xi[1] - xi[0] > 0
    assert (xi[1] - xi[0]) % (8 * nj) == 0          # the same whole count per node of every line


def test_stored_counts_match_the_script():
    with open(os.path.join(ROOT, "paper_1810_11103_gb300", "algorithmic_flops.json")) as f:
        stored = json.load(f)
    assert CF.vortex_counts() == stored["schemes"]
    assert CF.adjoint_counts() == stored["adjoint"]["schemes"]
    assert CF.three_d_counts() == stored["three_d"]["schemes"]


def test_midpoint_interpolation_counts():
    """One midpoint interpolation of a nodal quantity (Section 2.4), as the oracle writes it:
    the four-point Lagrange interpolant costs three products, three additions and one division
    (7), the six-point one six, five and one (12), the eight-point one eight, seven and one
    (16), and the two-point average an addition and a product (2)."""
    assert [O.count_mid_interp(s) for s in range(6)] == [7, 7, 12, 12, 16, 16]
    assert all(O.count_mid_interp(s, 1) == 2 for s in range(6))
    # the interface direction: two averages (2 each), |m| (two products, a sum, a square root),
    # two divisions
    assert O.count_char_dir() == 10


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_sweep_count_carries_two_interpolations_per_interface(scheme):
    """The xi sweep interpolates the two direction metrics at each of its n + 2 nmp - 1
    interfaces per line: switching the interpolation to the two-point average changes its count
    by exactly that many interpolations (linear weights: nothing else depends on the data)."""
    ni, nj = 20, 14
    nmp = 2 if scheme in (1, 3) else 1
    a = _parts(scheme, ni, nj, linear_weights=1)[1]
    b = _parts(scheme, ni, nj, linear_weights=1, interp=1)[1]
    assert a - b == nj * (ni + 2 * nmp - 1) * 2 * (O.count_mid_interp(scheme) - O.count_mid_interp(scheme, 1))
