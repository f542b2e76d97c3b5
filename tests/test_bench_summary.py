"""The bench line ends with a compact summary of every path, so that a reader who keeps only
the last ~1500 characters of the output (a log tail) still sees each precision's throughput,
roofline fraction and batching gain, the adjoint ratios and WENOIU7-1MP."""
import json
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _path(value, frac):
    return {"value": value, "ms_per_step": 1e3 / value, "e2e": {"value": 0.9 * value},
            "roofline": {"frac": frac, "frac_vs_nominal": 0.8 * frac, "kernel_ms": 1.2345678, "part": "FP64 part"},
            "per_block": {"value": 0.75 * value}}


def test_summary_is_compact_and_complete():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(precision="fp64")
    head = _path(255.123456, 0.7461234)
    others = {"fp32": _path(9762.0123, 0.479123), "mixed": _path(2841.5, 0.575)}
    others["mixed"].pop("per_block")
    adjoint = {"rhs_vjp_over_rhs": 3.7912, "rk3_step_vjp_over_rk3_step": 3.80123, "gradient_over_forward": 4.8012,
               "full_tape": {"gradient_over_forward": 3.8012}}
    seventh = {p: {"value": 181.23456, "roofline": {"frac": 0.9141}} for p in ("fp64", "fp32")}
    s = bench.summary(args, head, others, adjoint, seventh)
    text = json.dumps({"summary": s})
    assert len(text) < 1200
    assert s["fp64"]["value"] == 255.1 and s["fp64"]["frac"] == 0.746 and s["fp64"]["batch_gain"] == 1.33
    assert s["fp32"]["frac"] == 0.479 and s["fp32"]["per_block"] == 7322.0
    assert s["fp32_mixed"]["part"] == "FP64 part" and "per_block" not in s["fp32_mixed"]
    assert s["adjoint"]["grad_ckpt"] == 4.8 and s["wenoiu7"]["fp32"]["frac"] == 0.914
