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
    # the midpoint metric interpolation (two components) and the characteristic direction
    # inside those sweeps, per interface, over the n + 2 nmp - 1 interfaces of each line (a
    # solver may store them once per grid instead)
    nmp = 2 if scheme in (1, 3) else 1
    ifx = sum(b["x"].shape[0] * (b["x"].shape[1] + 2 * nmp - 1) for b in blocks)
    ife = sum(b["x"].shape[1] * (b["x"].shape[0] + 2 * nmp - 1) for b in blocks)
    return {"rhs_per_node": sum(tot) / nodes, "lambda_per_node": (lx + le) / nodes,
            "sweep_xi_per_node": sx / nodes, "sweep_eta_per_node": (se + fin) / nodes, "nodes": nodes,
            "mid_interp_per_interface": 2 * O.count_mid_interp(scheme),
            "char_dir_per_interface": O.count_char_dir(),
            "xi_interfaces_per_node": ifx / nodes, "eta_interfaces_per_node": ife / nodes}


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


def three_d_counts(n_work: int = 128):
    """Per-node operations of one three-dimensional right-hand side (and of its xi, eta and
    zeta sweeps) for an n_work^3 cube: a + b / n fits (every line of n nodes costs c1 n + c2)
    of 24^3 and 32^3 randomised periodic cubes carrying the three-dimensional vortex, as the
    bench's workload does (WENOIU5-1MP; with nonlinear weights the mapping's two sides differ
    by a few operations, so the fit is exact up to the data's branch mix)."""
    sizes = (24, 32)
    per = {}
    for n in sizes:
        x, y, z, pr = I.periodic_cube(n, 10.0, 0.2, seed=1810)
        q = I.vortex3(x, y, z, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0, 1.0), period=pr)
        cfg = dict(scheme=2, period=pr, bc=(0,) * 6)
        c = O.count_flops3(cfg, O.metrics3(cfg, x, y, z), q)
        per[n] = {k: v / x.size for k, v in c.items()}
    n0, n1 = sizes
    e = {}
    for k in ("rhs", "xi", "eta", "zeta"):
        b = (per[n0][k] - per[n1][k]) / (1.0 / n0 - 1.0 / n1)
        a = per[n1][k] - b / n1
        e[k + "_per_node"] = a + b / n_work
    return {NAMES[2]: e}


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
    res["three_d"] = {"workload": "128^3 randomised periodic cube (A = 0.2, seed 1810) with the three-dimensional "
                                  "vortex, from a + b/n fits of 24^3 and 32^3 cubes",
                      "how": "oracle three-dimensional path with the operation-counting scalar",
                      "schemes": three_d_counts()}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
