"""The integer double-to-float rounding of the float paths (`from_f64_int`, which keeps the
mixed path's conversions off the FP64 pipe) against the hardware conversion and against
numpy's round-to-nearest-even, through fsp_round_to_float: equal bit for bit on inputs in the
float normal range and above (ties, the overflow edge, infinities); NaN stays NaN; inputs below
the float normal range are flushed to signed zero by the integer rounding only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _cases():
    fmax = float(np.finfo(np.float32).max)
    ulp_top = 2.0 ** (127 - 23)                 # spacing of floats just below FLT_MAX
    one_ulp = 2.0 ** -23
    vals = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, -np.nan,
            fmax, -fmax, fmax + 0.25 * ulp_top, fmax + 0.5 * ulp_top, fmax + 0.75 * ulp_top, 1e300, -1e300,
            1.0 + 0.5 * one_ulp, 1.0 + 1.5 * one_ulp,                 # ties to even: down, up
            1.0 + 0.5 * one_ulp + 2.0 ** -60, -(1.0 + 1.5 * one_ulp),
            float(np.finfo(np.float32).tiny), 2.0 ** -126 * (1 - 2.0 ** -25)]
    rng = np.random.default_rng(1810)
    rnd = rng.standard_normal(4096) * 10.0 ** rng.uniform(-30, 30, 4096)
    return np.concatenate([np.array(vals, dtype=np.float64), rnd])


def test_integer_rounding_matches_the_hardware(F):
    x = _cases()
    a, b = F.round_to_float(torch.as_tensor(x, device="cuda"))
    torch.cuda.synchronize()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    nan = np.isnan(x)
    assert np.isnan(a[nan]).all() and np.isnan(b[nan]).all()
    normal_or_big = ~nan & ((np.abs(x) >= np.finfo(np.float32).tiny) | (x == 0))
    assert np.array_equal(a[normal_or_big].view(np.uint32), ref[normal_or_big].view(np.uint32))
    assert np.array_equal(b[normal_or_big].view(np.uint32), ref[normal_or_big].view(np.uint32))
    tiny = ~nan & ~normal_or_big
    assert tiny.any()
    assert (a[tiny] == 0).all() and np.array_equal(np.signbit(a[tiny]), np.signbit(x[tiny]))


def test_integer_widening_matches_the_hardware(F):
    """to_f64_int (the mixed path's float-to-double widening, integer operations only): bit for
    bit the hardware's on signed zeros, normals across the whole exponent range, the float
    extremes and infinities; NaN stays NaN; subnormals become signed zero."""
    f32 = np.finfo(np.float32)
    rng = np.random.default_rng(1103)
    vals = np.array([0.0, -0.0, 1.0, -1.0, f32.max, -f32.max, f32.tiny, -f32.tiny, f32.tiny / 2, -f32.tiny / 8,
                     2.0 ** -149, np.inf, -np.inf, np.nan], dtype=np.float32)
    rnd = (rng.standard_normal(8192) * 10.0 ** rng.uniform(-44, 38, 8192)).astype(np.float32)
    bits = rng.integers(0, 2 ** 32, 8192, dtype=np.uint64).astype(np.uint32).view(np.float32)   # every pattern kind
    x = np.concatenate([vals, rnd, bits])
    a, b = F.widen_to_double(torch.as_tensor(x, device="cuda"))
    torch.cuda.synchronize()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    nan = np.isnan(x)
    sub = (x != 0) & (np.abs(x) < f32.tiny)
    assert np.isnan(a[nan]).all() and sub.any()
    assert (a[sub] == 0).all() and np.array_equal(np.signbit(a[sub]), np.signbit(x[sub]))
    keep = ~nan & ~sub
    assert np.array_equal(a[keep].view(np.uint64), b[keep].view(np.uint64))
    assert np.array_equal(b[~nan], x[~nan].astype(np.float64))


def test_fp64_reciprocal_within_ulps_of_ieee(F):
    """rcp_nr (the hardware seed and one third-order Householder step), used by every FP64
    kernel for densities, J^-1 and weight sums: within 2 ulps of the correctly rounded 1/x
    over normal operands of both signs across the exponent range (the seed flushes
    subnormals, so reciprocals of numbers beyond 2^1022 are not taken); rsq_nr, used for
    sound speeds and metric norms, within 3 ulps of 1/sqrt(x) (itself two roundings)."""
    rng = np.random.default_rng(1810)
    mag = 2.0 ** rng.uniform(-1000, 1000, 200000)
    x = mag * np.where(rng.random(200000) < 0.5, -1.0, 1.0)
    x = np.concatenate([x, [1.0, 3.0, 0.1, 1.0 / 3.0, 2.0 ** -1000, 1.5 * 2.0 ** 1000]])
    a, b, c, d = (t.cpu().numpy() for t in F.reciprocal_check(torch.as_tensor(x, device="cuda")))
    assert np.array_equal(b, 1.0 / x)
    ulp = np.spacing(np.abs(b))
    assert (np.abs(a - b) <= 2 * ulp).all(), float((np.abs(a - b) / ulp).max())
    # rsq_nr (the hardware seed and one third-order step) for the positive operands
    pos = x > 0
    ref = 1.0 / np.sqrt(x[pos])
    assert np.array_equal(d[pos], ref) and (c[~pos] == 0).all()
    ulp = np.spacing(ref)
    assert (np.abs(c[pos] - ref) <= 3 * ulp).all(), float((np.abs(c[pos] - ref) / ulp).max())
