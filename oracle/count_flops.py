"""Writes paper_1810_11103_gb300/algorithmic_flops.json: floating-point operations of one
right-hand side per node, counted by running the oracle with an operation-counting scalar
(each + - * / sqrt counts one; a fused multiply-add is two).  Used as the algorithmic
work of the roofline.  The adjoint's count comes from the oracle's reverse mode: the forward
right-hand side, the partial derivatives its divisions and square roots need, and the dense
reverse sweep of its tape (one operation per operand edge whose partial is +-1, two for any
other).  Run: python -m oracle.count_flops
"""
import json
import os

import numpy as np

from . import oracle as O
from paper_1810_11103_gb300 import inputs as I

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1810_11103_gb300", "algorithmic_flops.json")


def cylinder_counts(scheme):
    """Per-node flops of the 64-block cylinder workload: every block counted on its own
    with linked faces read as transmissive (the per-interface arithmetic does not depend
    on where a ghost state comes from)."""
    blocks, states, free = I.cylinder_blocks()
    tot = [0, 0, 0, 0, 0]
    nodes = 0
    for b, q in zip(blocks, states):
        bc = [1 if c == I.LINK else c for c in b["bc"]]
        cfg = dict(scheme=scheme, bc=bc, bc_state=[list(free)] * 4)
        M = O.metrics(cfg, b["x"], b["y"])
        parts = O.count_flops_parts(cfg, M, q)
        tot = [t + p for t, p in zip(tot, parts)]
        nodes += b["x"].size
    lx, sx, le, se, fin = tot
    return {"rhs_per_node": sum(tot) / nodes, "lambda_per_node": (lx + le) / nodes,
            "sweep_xi_per_node": sx / nodes, "sweep_eta_per_node": (se + fin) / nodes, "nodes": nodes}


NAMES = ["WENOIU3-1MP", "WENOIU3-2MP", "WENOIU5-1MP", "WENOIU5-2MP", "WENOIU7-1MP"]


def vortex_counts():
    """Per-node flops of every scheme on the 256 x 256 periodic vortex."""
    x, y, per = I.periodic_square(256, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    n = x.size
    out = {}
    for s in range(5):
        cfg = dict(scheme=s, period=per)
        M = O.metrics(cfg, x, y)
        lx, sx, le, se, fin = O.count_flops_parts(cfg, M, q)
        out[NAMES[s]] = {
            "rhs_per_node": (lx + sx + le + se + fin) / n,
            "lambda_per_node": (lx + le) / n,
            "sweep_xi_per_node": sx / n,
            "sweep_eta_per_node": (se + fin) / n,
        }
    return out


def adjoint_counts(n_work: int = 512):
    """Per-node operations of one right-hand-side adjoint for the adjoint workload's
    n_work x n_work grid.  Every line of n nodes costs c1 n + c2 (its interfaces include a
    halo), so on an n x n periodic grid the per-node count is a + b / n (exactly so with linear
    weights; the two sides of the mapping differ by a few operations, so with nonlinear weights
    up to the data's branch mix); it is counted on 48 x 48 and 64 x 64 periodic vortices (the
    adjoint workload's epsilon) and evaluated at n_work."""
    sizes = (48, 64)
    per = {}
    for n in sizes:
        x, y, pr = I.periodic_square(n, 10.0, 0.2, seed=1810)
        q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
        for s in range(4):
            cfg = dict(scheme=s, period=pr, eps=1e-6)
            M = O.metrics(cfg, x, y)
            c = O.count_vjp_flops(cfg, M, q)
            per[(n, s)] = {k: c[k] / x.size for k in ("forward", "partials", "reverse")}
    out = {}
    n0, n1 = sizes
    for s in range(4):
        e = {}
        for k in ("forward", "partials", "reverse"):
            b = (per[(n0, s)][k] - per[(n1, s)][k]) / (1.0 / n0 - 1.0 / n1)
            a = per[(n1, s)][k] - b / n1
            e[k + "_per_node"] = a + b / n_work
        e["vjp_per_node"] = e["forward_per_node"] + e["partials_per_node"] + e["reverse_per_node"]
        out[NAMES[s]] = e
    return out


def main():
    res = {"workload": "periodic vortex 256x256, randomised grid A=0.2, seed 1810",
           "how": "oracle with an operation-counting scalar; + - * / sqrt = 1 flop each",
           "schemes": vortex_counts()}
    names = NAMES
    res["cylinder64"] = {"workload": "64-block cylinder (seed 1812), linked faces counted as transmissive",
                         "schemes": {names[s]: cylinder_counts(s) for s in (2, 4)}}
    res["adjoint"] = {"workload": "512x512 lines (the shock-vortex adjoint workload), from exact a + b/n fits of "
                                  "48x48 and 64x64 periodic vortices, randomised grid A=0.2, seed 1810, eps 1e-6",
                      "how": "oracle reverse mode: forward + partial derivatives + dense reverse sweep",
                      "schemes": adjoint_counts()}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
