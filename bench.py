#!/usr/bin/env python
"""Benchmark of the WENOIU free-stream-preserving Euler right-hand side on GB300.

Workload (default "cylinder64"): supersonic flow (Mach 4) around a cylinder on 64 body-fitted
blocks of uneven sizes (5.9 M nodes, 30 % of the blocks randomised), WENOIU5-1MP.  One step
= one TVD-RK3 step of every block (three right-hand sides), launched as one captured CUDA
graph through fsp_batch_rk3_step.  Metric: Mcell-RHS/s = nodes x right-hand sides / second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--workload cylinder64|vortex256] [--precision fp64|fp32|mixed]
                    [--no-all-precisions] [--no-cpu-baseline] [--accuracy none|quick|full]

The headline `value` is the FP64 path.  Beside it: the FP32 and mixed FP32/FP64 paths of the
same workload ("fp32", "fp32_mixed"), each with its own roofline, and the same FP64 and FP32
steps as loops of per-block fsp_rk3_step calls ("per_block_fp64", "fp32.per_block", links read
as transmissive).  With --accuracy quick|full ("accuracy"): final-time density errors of each
precision on the 256 x 256 vortex (full adds the 1024 x 1024 Riemann problem) and the
free-stream residual.  The line ends with "summary", the compact figures of every path.
Under torchrun every rank runs the workload on its own GPU (independent problems, weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-RHS/s 2-D Euler WENO5 FP64 vs FP32 batched, % roofline; adjoint/fwd ratio"
UNIT = "Mcell-RHS/s"
SCHEME_NAMES = ["WENOIU3-1MP", "WENOIU3-2MP", "WENOIU5-1MP", "WENOIU5-2MP", "WENOIU7-1MP"]
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}
DTYPES = {"fp64": "f64", "fp32": "f32", "mixed": "f32+f64"}
L2_FLUSH_BYTES = 256 << 20   # larger than the 129 MB L2
LINK = 5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="cylinder64", choices=["cylinder64", "vortex256"])
    ap.add_argument("--scheme", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS))
    ap.add_argument("--all-precisions", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure the other two precisions and report them beside the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint cost measurement")
    ap.add_argument("--three-d", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure the three-dimensional path (fsp3_*) on a 128^3 randomised periodic cube, "
                         "WENOIU5-1MP, FP64")
    ap.add_argument("--seventh", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure WENOIU7-1MP (the Appendix's seventh-order scheme) on the same workload, "
                         "FP64 and FP32")
    ap.add_argument("--accuracy", choices=["none", "quick", "full"], default="none",
                    help="final-time errors per precision: quick = the 256 x 256 vortex over one period and "
                         "the free-stream residual; full adds the 1024 x 1024 Riemann problem to t = 0.3")
    ap.add_argument("--tune-table", default=None,
                    help="text file of tile choices for fsp_batch_tune: a workload found there takes the "
                         "stored variants without timing, otherwise the timed choice is appended (lets a "
                         "run under a profiler launch the kernels an unprofiled run chose)")
    ap.add_argument("--profile-tiles", default="2,1",
                    help="profiling run: tile shape variants 'vx,ve' of the xi and eta passes (the tuner's "
                         "choice on this workload), set without timing")
    ap.add_argument("--profile-dir", type=int, default=0, choices=[0, 1],
                    help="profiling run: the direction whose batched sweep is launched three times")
    ap.add_argument("--profile", choices=list(PRECISIONS) + ["adjoint", "probe", "three_d"], default=None,
                    help="profiling run for ncu: build the cylinder batch in this precision, evaluate one "
                         "right-hand side, launch one direction's batched sweep three times, then take one "
                         "RK3 step; 'adjoint': three "
                         "fsp_rhs_vjp calls on the 512 x 512 shock-vortex case; 'probe': the FP64 and the "
                         "FP32 FMA probe once each, as the bench launches them; 'three_d': the 3-D metrics and "
                         "one 3-D right-hand side of the bench's 128^3 cube; no timing")
    ap.add_argument("--per-block", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the FP64 and FP32 steps as loops of per-block fsp_rk3_step calls")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------
def cylinder_workload():
    """64 blocks around a cylinder of diameter one (seed 1812): 8 angular columns x 8 radial
    rows, sizes 64..512 x 64..384, slip wall, far field at Mach 4, 30 % randomised blocks."""
    from paper_1810_11103_gb300 import inputs as I
    return I.cylinder_blocks()


def vortex_workload(n=256):
    from paper_1810_11103_gb300 import inputs as I
    x, y, per = I.periodic_square(n, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    return x, y, per, q


def workload_config(args, nodes, nblocks):
    if args.workload == "cylinder64":
        return {"workload": f"Mach 4 cylinder, {nblocks} linked blocks of uneven sizes (seed 1812), "
                            f"{SCHEME_NAMES[args.scheme]}, TVD-RK3",
                "nodes": nodes, "blocks": nblocks, "scheme": SCHEME_NAMES[args.scheme], "precision": args.precision,
                "step": "one RK3 step of every block = 3 right-hand sides, one captured CUDA graph",
                "l2": "inputs larger than L2 (state and metrics > 300 MB); no flush"}
    return {"workload": f"periodic isentropic vortex 256x256, randomised grid +-0.2h, {SCHEME_NAMES[args.scheme]}",
            "nodes": nodes, "blocks": 1, "scheme": SCHEME_NAMES[args.scheme], "precision": args.precision,
            "step": "one RK3 step = 3 right-hand sides",
            "l2": "flushed between timed steps (256 MiB write outside the events)"}


# the sources the batched sweep kernels (the roofline kernels) are built from
SWEEP_SOURCES = ("sweep.cuh", "fsp_device.cuh", "fsp_internal.h", "batch_fp64.cu", "batch_fp32.cu", "batch_mixed.cu")


def source_hash():
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_1810_11103_gb300", "csrc")
    for f in SWEEP_SOURCES:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def algorithmic_flops(args):
    with open(os.path.join(ROOT, "paper_1810_11103_gb300", "algorithmic_flops.json")) as f:
        d = json.load(f)
    if args.workload == "cylinder64":
        return d["cylinder64"]["schemes"][SCHEME_NAMES[args.scheme]]
    return d["schemes"][SCHEME_NAMES[args.scheme]]


def traffic_of(args, prec, variant, direction=0):
    """DRAM bytes of one launch of the xi (direction 0) or eta (1) sweep in tile variant
    `variant`, from an ncu capture of the current kernel sources (None if there is none)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        entries = json.load(f)
    for tr in entries if isinstance(entries, list) else [entries]:
        if (tr.get("source_hash") == source_hash() and tr.get("workload") == args.workload
                and tr.get("scheme") == args.scheme and tr.get("precision") == prec
                and tr.get("variant") == variant and tr.get("dir", 0) == direction):
            return tr.get("bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi clock and throttle samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)   # let the first samples arrive before the timed region
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [a.strip() for a in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU baseline and the reference arm: the oracle, as it stands, on one host core
# ------------------------------------------------------------------------------------------
def oracle_sample(args):
    """(cfg, metrics, state, nodes, description) of the bounded sample the oracle is timed
    on: for the cylinder, its first block (512 x 384) with linked faces read as transmissive
    (the same arithmetic per node); for the vortex, the whole 256 x 256 block."""
    import numpy as np
    import oracle as O
    if args.workload == "cylinder64":
        blocks, states, free = cylinder_workload()
        b = blocks[0]
        cfg = dict(scheme=args.scheme, bc=[1 if c == LINK else c for c in b["bc"]],
                   bc_state=np.tile(free, (4, 1)))
        M = O.metrics(cfg, b["x"], b["y"])
        return cfg, M, states[0], b["x"].size, f"block 0 ({b['x'].shape[1]}x{b['x'].shape[0]}) of the cylinder"
    x, y, per, q = vortex_workload()
    cfg = dict(scheme=args.scheme, period=per)
    return cfg, O.metrics(cfg, x, y), q, x.size, "the 256x256 vortex block"


def cpu_baseline(args, seconds=12.0):
    import oracle as O
    cfg, M, q, nodes, what = oracle_sample(args)
    t0 = time.perf_counter()
    k = 0
    while True:
        O.rhs(cfg, M, q)
        k += 1
        t = time.perf_counter() - t0
        if t > seconds:
            break
    out = {"value": nodes * k / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{k} right-hand sides of {what} (oracle, one thread)"}
    if args.workload == "cylinder64":
        out["all_cores"] = cpu_all_cores(args)
    return out


def _oracle_block_rhs(job):
    """One worker process: the oracle's right-hand side of one cylinder block (linked faces
    read as transmissive), timed after its metrics are built."""
    scheme, k = job
    import numpy as np
    import oracle as O
    blocks, states, free = cylinder_workload()
    b = blocks[k]
    cfg = dict(scheme=scheme, bc=[1 if c == LINK else c for c in b["bc"]], bc_state=np.tile(free, (4, 1)))
    M = O.metrics(cfg, b["x"], b["y"])
    t0 = time.perf_counter()
    O.rhs(cfg, M, states[k])
    return b["x"].size, time.perf_counter() - t0


def cpu_all_cores(args):
    """The oracle on every host core at once: one right-hand side of each of the 64 cylinder
    blocks, spread over a pool of worker processes (spawned: this process already holds a CUDA
    context).  Rate = cores x (nodes / seconds summed over the blocks), the throughput with
    every core busy."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    nblocks = len(cylinder_workload()[0])
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_block_rhs, [(args.scheme, k) for k in range(nblocks)], chunksize=1)
    nodes = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    return {"value": cores * nodes / busy / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one right-hand side of each of the {nblocks} cylinder blocks ({nodes} nodes), "
                      f"{cores} worker processes"}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle as O
    O.build()
    cfg, M, q, nodes, what = oracle_sample(args)
    if args.workload == "cylinder64":
        blocks = cylinder_workload()[0]
        job_nodes, nblocks = sum(b["x"].size for b in blocks), len(blocks)
    else:
        job_nodes, nblocks = nodes, 1
    for _ in range(args.warmup):
        O.rhs(cfg, M, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rhs(cfg, M, q)
    t = time.perf_counter() - t0
    value = nodes * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, job_nodes, nblocks),
            "reference_step": f"one right-hand side of {what} (oracle, one host thread); the rate is per "
                              f"node and right-hand side, as on the GPU arm",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"a bounded sample of the workload: {args.steps} right-hand sides of {what} "
                                       f"(oracle, one host thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# GPU measurement
# ------------------------------------------------------------------------------------------
def job_rhs(nodes, steps, world):
    """Right-hand sides x nodes of the whole job: every rank advances its own copy of the
    workload (weak scaling), three right-hand sides per RK3 step; divided by the slowest
    rank's time this is the job's Mcell-RHS/s."""
    return nodes * 3 * steps * world


class Ctx:
    def __init__(self, torch, fsp, dist, dev, world):
        self.torch, self.fsp, self.dist, self.dev, self.world = torch, fsp, dist, dev, world
        self.stream = torch.cuda.current_stream() if dev.type == "cuda" else None
        self.flush = None

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()
        if self.dev.type == "cuda":
            self.torch.cuda.synchronize()

    def timed(self, body, reps, flush=False):
        torch = self.torch
        if flush and self.flush is None:
            self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=self.dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        self.barrier()
        for a, b in ev:
            if flush:
                self.flush.zero_()
            a.record(self.stream)
            body()
            b.record(self.stream)
        self.barrier()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    def sm_count(self):
        return int(self.torch.cuda.get_device_properties(self.dev).multi_processor_count)

    def peak(self, prec):
        """FMA rate of the path's pipe measured by fsp_fma_peak (8 resident 256-thread CTAs
        per SM of this device, 8 independent FMA chains per thread), in TFLOP/s."""
        fsp, torch = self.fsp, self.torch
        pipe = 0 if prec == "fp64" else 1
        blocks, iters = self.sm_count() * 8, 4096 if pipe == 0 else 65536
        sink = torch.empty(blocks * 256, dtype=torch.float64 if pipe == 0 else torch.float32, device=self.dev)
        fsp.fma_peak(pipe, blocks, iters, sink)
        t = self.timed(lambda: fsp.fma_peak(pipe, blocks, iters, sink), 3) / 3
        return 2.0 * 8 * iters * blocks * 256 / t / 1e12, ("FP64" if pipe == 0 else "FP32")

    def nominal(self, prec, mhz):
        """Nominal FMA rate at the SM clock sampled during the run: SMs x FMA lanes per SM per
        clock x 2 flops x clock (FP64: 2 lanes per SM on this part, the 1.25 TFLOP/s of its
        data sheet at 2.07 GHz; FP32: 128 lanes)."""
        lanes = 2 if prec == "fp64" else 128
        return self.sm_count() * lanes * 2.0 * (mhz or 2070.0) * 1e6 / 1e12

    def max_over_ranks(self, *vals):
        if self.world == 1:
            return vals
        t = self.torch.tensor(vals, dtype=self.torch.float64, device=self.dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return tuple(float(v) for v in t)


def launches_per_step(args, head):
    """Kernels of one batched RK3 step: per stage an xi and an eta sweep, plus the line maxima of
    every stage, or of the first only when the marching eta pass takes them (not in mixed
    precision), plus the midpoint metrics once per step (FP64 and mixed batches); the vortex
    workload's single-block step always has three per stage."""
    if args.workload != "cylinder64":
        return 9
    fused = (head.get("tiles") or {}).get("eta", {}).get("variant") == 3 and args.precision != "mixed"
    return (7 if fused else 9) + (args.precision != "fp32")


def measure_cylinder(args, prec, C, per_block=False):
    import numpy as np
    torch, fsp = C.torch, C.fsp
    blocks, states, free = cylinder_workload()
    cfgd = dict(scheme=args.scheme, precision=PRECISIONS[prec], bc_state=np.tile(free, (4, 1)))
    cfg = fsp.Config.from_dict(cfgd)
    bt = fsp.Batch(cfg, blocks, states, device=C.dev)
    bt.metrics()
    # tile shapes chosen by timing each variant's pass on this batch (fsp_batch_tune)
    tiles = {d: dict(zip(("variant", "lines", "outputs_per_line"), t)) for d, t in zip(("xi", "eta"), bt.tune(args.tune_table))}
    nodes = sum(b["x"].size for b in blocks)
    # a stable step: CFL 0.3 on the initial state, from the per-block CFL rate
    dts = []
    for k, b in enumerate(blocks):
        cb = fsp.Config.from_dict(dict(cfgd, bc=[1 if c == LINK else c for c in b["bc"]]))
        dts.append(float(fsp.cfl_dt(cb, bt.M[k], bt.Q[k], 0.3).item()))
    dt = min(dts)
    bt.capture_graph(dt)
    for _ in range(args.warmup):
        bt.rk3_step(dt)
    clocks = ClockSampler(C.dev.index or 0)
    clocks.start()
    t_dev = C.timed(lambda: bt.rk3_step(dt), args.steps)
    clk = clocks.stop()
    # end to end through one C-ABI call (fsp_batch_rk3_step_host): every block's state from
    # pinned host memory, the step, the states back to pinned host memory (the states lie in
    # one buffer, so the library makes one copy each way)
    host_in = bt.Qflat.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def e2e():
        bt.rk3_step_host(dt, host_in, host_out)
    e2e()
    t_e2e = C.timed(e2e, args.steps)
    state_bytes = host_in.numel() * host_in.element_size()
    # the dominant kernel alone: the xi sweep of every block (one launch)
    bt.Qflat.copy_(host_in)
    bt.rhs()
    D = [torch.empty(q.shape, dtype=torch.float32 if prec == "fp32" else torch.float64, device=C.dev) for q in bt.Q]
    bt.flux_difference(0, D)
    t_k = C.timed(lambda: bt.flux_difference(0, D), 20) / 20
    bt.flux_difference(1, D)
    t_e = C.timed(lambda: bt.flux_difference(1, D), 20) / 20
    peak, pipe = C.peak(prec)
    t_dev, t_e2e = C.max_over_ranks(t_dev, t_e2e)
    fl = algorithmic_flops(args)
    # FP64 and mixed batches store the midpoint metrics (FP64 also the characteristic direction)
    # once per step (mid_batch_kernel) and the marching passes read them: that work leaves the
    # passes' counts and enters the step's once instead of three times
    mid_if = fl["mid_interp_per_interface"] if prec != "fp32" else 0
    mid_if += fl["char_dir_per_interface"] if prec == "fp64" else 0   # FP64 reads the direction too
    mid_xi = fl["xi_interfaces_per_node"] * mid_if * (tiles["xi"]["variant"] == 3)
    mid_eta = fl["eta_interfaces_per_node"] * mid_if * (tiles["eta"]["variant"] == 3)
    xi_fl = fl["sweep_xi_per_node"] - mid_xi
    eta_fl = fl["sweep_eta_per_node"] - 4.0 - mid_eta
    step_fl = 3 * fl["rhs_per_node"] - 2 * (mid_xi + mid_eta)
    rhs_total = job_rhs(nodes, args.steps, C.world)
    nom = C.nominal(prec, clk.get("sm_mhz"))

    def pass_roof(d, fl_node, t):
        var = tiles["xi" if d == 0 else "eta"]["variant"]
        name = (("march_batch_kernel xi (marching warps)" if var == 3 else "sweep_batch_kernel xi") if d == 0 else
                ("march_eta_batch_kernel eta (marching CTAs)" if var == 3 else "sweep_batch_kernel eta"))
        a = fl_node * nodes / t / 1e12
        return {"kernel": name + f", all 64 blocks (fsp_batch_flux_difference dir {d})", "kernel_ms": 1e3 * t,
                "flops_per_node": fl_node, "achieved": a, "frac": a / peak, "frac_vs_nominal": a / nom,
                "traffic": traffic_of(args, prec, var, d)}
    passes = {"xi": pass_roof(0, xi_fl, t_k), "eta": pass_roof(1, eta_fl, t_e)}
    # the roofline kernel: the longer of the two passes, each timed alone (one launch over all
    # blocks); the other beside it
    dom = "eta" if t_e > t_k else "xi"
    roof = {"bound": "alu", **passes[dom], "direction": dom, "peak": peak, "unit": "TFLOP/s",
            "peak_source": f"{pipe} FMA probe (fsp_fma_peak) in this run, same clocks",
            "nominal_peak": nom, "units_per_launch": nodes,
            "xi": passes["xi"], "eta": passes["eta"],
            # the whole step against the same peak
            "step_frac": step_fl * nodes / (t_dev / args.steps) / 1e12 / peak,
            "midpoint_metrics": ({"flops_per_node_per_step": mid_xi + mid_eta,
                                  "how": "midpoint metrics" + (" and characteristic direction" if prec == "fp64" else "")
                                         + " per interface once per step by mid_batch_kernel; left out of the "
                                           "passes' counts"} if mid_if else None)}
    if prec == "mixed":
        roof = mixed_roofline(args, C, roof, passes[dom]["flops_per_node"], nodes, t_e if dom == "eta" else t_k,
                              clk.get("sm_mhz"), hoisted=mid_xi > 0)
    out = {
        "value": rhs_total / t_dev / 1e6, "ms_per_step": 1e3 * t_dev / args.steps, "nodes": nodes,
        "nblocks": len(blocks),
        "e2e": {"value": rhs_total / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "call": "fsp_batch_rk3_step_host (pinned host buffers)"},
        "roofline": roof,
        "clocks": clk,
        "tiles": tiles,
    }
    if per_block:
        # the same step as a loop of single-block calls (links read as transmissive)
        cbs, wss = [], []
        for k, b in enumerate(blocks):
            cb = fsp.Config.from_dict(dict(cfgd, bc=[1 if c == LINK else c for c in b["bc"]]))
            cbs.append(cb)
            wss.append(fsp.workspace(cb, bt.Q[k]))

        def loop():
            for k in range(len(blocks)):
                fsp.rk3_step(cbs[k], bt.M[k], bt.Q[k], dt, ws=wss[k])
        loop()
        reps = max(3, args.steps // 4)
        t_loop = C.timed(loop, reps)
        out["per_block"] = {"value": nodes * 3 * reps / t_loop / 1e6, "unit": UNIT,
                            "ms_per_step": 1e3 * t_loop / reps,
                            "how": "64 fsp_rk3_step calls per step, one block each, eager launches"}
    bt.close()
    return out


# FP64 operations per node of one direction in the mixed path (FP32 state, projection, WENO,
# Cartesian fluxes and dissipative part; double metric products, central combination and
# difference), counted from its formulas with a fused multiply-add as two: node products
# mx E + my F (4 x 3), midpoint metric interpolation (2 x 9 six-point, 2 x 5 four-point, 2 x 12
# eight-point),
# midpoint products (one mean flux, 4 x 3; two-midpoint schemes both sides, 4 x 6), central
# combination of node pairs and midpoint terms, double + float parts and the difference (4 + 4).
MIXED_FP64_FLOPS = {0: 70, 1: 86, 2: 90, 3: 106, 4: 108}
# of which the midpoint metric interpolation, which a batch with stored midpoint metrics no
# longer does in the passes
MIXED_FP64_MID_FLOPS = {0: 10, 1: 10, 2: 18, 3: 18, 4: 24}


def mixed_roofline(args, C, roof, flops_node, nodes, t_k, mhz, hoisted=False):
    """Roofline of the mixed path: t_roof = max(FP32 flops / FP32 peak, FP64 flops / FP64
    peak); the FP64 part bounds it.  The FP32 part is the rest of the algorithmic count."""
    f64 = MIXED_FP64_FLOPS[args.scheme] - (MIXED_FP64_MID_FLOPS[args.scheme] if hoisted else 0)
    f32 = flops_node - f64
    p64, _ = C.peak("fp64")
    p32 = roof["peak"]
    t32, t64 = f32 * nodes / (p32 * 1e12), f64 * nodes / (p64 * 1e12)
    n32, n64 = C.nominal("fp32", mhz), C.nominal("fp64", mhz)
    part32 = {"flops_per_node": f32, "achieved": f32 * nodes / t_k / 1e12, "peak": p32,
              "frac": f32 * nodes / t_k / 1e12 / p32, "nominal_peak": n32,
              "frac_vs_nominal": f32 * nodes / t_k / 1e12 / n32}
    part64 = {"flops_per_node": f64, "achieved": f64 * nodes / t_k / 1e12, "peak": p64,
              "frac": f64 * nodes / t_k / 1e12 / p64, "nominal_peak": n64,
              "frac_vs_nominal": f64 * nodes / t_k / 1e12 / n64}
    head, other = (part64, part32) if t64 >= t32 else (part32, part64)
    out = dict(roof)
    # both sweeps against the bounding part as well (the FP64 operations of each; the float line
    # maxima are left out of the bound)
    for d in ("xi", "eta"):
        td = roof[d]["kernel_ms"] / 1e3
        out[d] = dict(roof[d], flops_per_node=f64, frac=f64 * nodes / td / 1e12 / p64,
                      achieved=f64 * nodes / td / 1e12, frac_vs_nominal=f64 * nodes / td / 1e12 / n64,
                      part="FP64 part")
    out["step_frac"] = None
    out.update({"bound": "alu", "achieved": head["achieved"], "peak": head["peak"], "frac": head["frac"],
                "nominal_peak": head["nominal_peak"], "frac_vs_nominal": head["frac_vs_nominal"],
                "flops_per_node": head["flops_per_node"],
                "part": "FP64 part" if head is part64 else "FP32 part",
                "peak_source": ("FP64" if head is part64 else "FP32") + " FMA probe (fsp_fma_peak) in this run",
                "other_part": other, "t_roof_ms": 1e3 * max(t32, t64)})
    return out


def measure_vortex(args, prec, C):
    torch, fsp = C.torch, C.fsp
    x, y, per, q = vortex_workload()
    cfg = fsp.Config.from_dict(dict(scheme=args.scheme, precision=PRECISIONS[prec], period=per))
    M = fsp.metrics(cfg, torch.as_tensor(x, device=C.dev), torch.as_tensor(y, device=C.dev))
    sdt = torch.float64 if prec == "fp64" else torch.float32
    Q = torch.as_tensor(q, dtype=sdt, device=C.dev)
    ws = fsp.workspace(cfg, Q)
    dt = float(fsp.cfl_dt(cfg, M, Q, 0.5, ws=ws).item())
    nodes = x.size
    for _ in range(args.warmup):
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
    clocks = ClockSampler(C.dev.index or 0)
    clocks.start()
    t_dev = C.timed(lambda: fsp.rk3_step(cfg, M, Q, dt, ws=ws), args.steps, flush=True)
    clk = clocks.stop()
    Qh = torch.as_tensor(q, dtype=sdt).pin_memory()
    Qout = torch.empty_like(Qh).pin_memory()

    def e2e():
        Q.copy_(Qh, non_blocking=True)
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
        Qout.copy_(Q, non_blocking=True)
    e2e()
    t_e2e = C.timed(e2e, args.steps, flush=True)
    lx, le = fsp.line_lambda(cfg, M, Q)
    D = torch.empty(Q.shape, dtype=torch.float32 if prec == "fp32" else torch.float64, device=C.dev)
    fsp.flux_difference(cfg, M, Q, lx, 0, 0, out=D)
    t_k = C.timed(lambda: fsp.flux_difference(cfg, M, Q, lx, 0, 0, out=D), 20, flush=True) / 20
    peak, pipe = C.peak(prec)
    t_dev, t_e2e = C.max_over_ranks(t_dev, t_e2e)
    fl = algorithmic_flops(args)
    achieved = fl["sweep_xi_per_node"] * nodes / t_k / 1e12
    rhs_total = job_rhs(nodes, args.steps, C.world)
    sb = Q.numel() * Q.element_size()
    nom = C.nominal(prec, clk.get("sm_mhz"))
    return {
        "value": rhs_total / t_dev / 1e6, "ms_per_step": 1e3 * t_dev / args.steps, "nodes": nodes, "nblocks": 1,
        "e2e": {"value": rhs_total / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": sb, "d2h_bytes_per_step": sb},
        "roofline": {"bound": "alu", "kernel": "sweep_kernel xi (fsp_flux_difference dir 0)", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic_of(args, prec, -1),
                     "peak_source": f"{pipe} FMA probe (fsp_fma_peak) in this run, same clocks",
                     "nominal_peak": nom, "frac_vs_nominal": achieved / nom,
                     "flops_per_node": fl["sweep_xi_per_node"], "units_per_launch": nodes,
                     "kernel_ms": 1e3 * t_k},
        "clocks": clk,
    }


def measure_adjoint(args, C, nsteps=200, every=14):
    """Adjoint cost on the shock-vortex case (512 x 512 stretched grid, Mach 1.1 shock plus
    vortex, WENOIU5-1MP, FP64): each adjoint entry point against its forward, and the
    gradient of the pressure functional over a 200-step march at CFL 0.5 with checkpoints
    every 14 steps (forward with checkpoints + reverse sweep with segment recompute)
    against the plain 200-step march."""
    import numpy as np
    torch, fsp = C.torch, C.fsp
    from paper_1810_11103_gb300 import autograd as AD
    from paper_1810_11103_gb300 import inputs as I
    from paper_1810_11103_gb300 import objectives as OBJ
    x, y = I.shock_vortex_grid(512)
    q0 = I.shock_vortex_state(x, y)
    bc, st = I.shock_vortex_bc()
    cfg = fsp.Config.from_dict(dict(scheme=args.scheme, bc=bc, bc_state=st, eps=1e-6))
    gx, gy = torch.as_tensor(x, device=C.dev), torch.as_tensor(y, device=C.dev)
    Q = torch.as_tensor(q0, device=C.dev)
    M = fsp.metrics(cfg, gx, gy)
    ws, vws = fsp.workspace(cfg, Q), fsp.vjp_workspace(cfg, Q)
    R, Qb, Mb = torch.empty_like(Q), torch.zeros_like(Q), torch.zeros_like(M)
    g = torch.as_tensor(I.smooth_field(x.shape, 7), device=C.dev).expand(4, -1, -1).contiguous()
    dts, _ = AD.cfl_schedule(cfg, M, Q, nsteps, 0.5)
    dt = dts[0]
    Qs = Q.clone()
    reps = 20
    for f in (lambda: fsp.rhs(cfg, M, Q, out=R, ws=ws), lambda: fsp.rhs_vjp(cfg, M, Q, g, Qb, Mb, ws=vws)):
        f()
    t_rhs = C.timed(lambda: fsp.rhs(cfg, M, Q, out=R, ws=ws), reps, flush=True) / reps
    t_rhs_vjp = C.timed(lambda: fsp.rhs_vjp(cfg, M, Q, g, Qb, Mb, ws=vws), reps, flush=True) / reps
    t_rk3 = C.timed(lambda: fsp.rk3_step(cfg, M, Qs, dt, ws=ws), reps, flush=True) / reps
    t_rk3_vjp = C.timed(lambda: fsp.rk3_step_vjp(cfg, M, Q, dt, Qb, Mb, ws=vws), reps, flush=True) / reps
    win = OBJ.window_of(x)

    def march():
        Qm = Q.clone()
        for d in dts:
            fsp.rk3_step(cfg, M, Qm, d, ws=ws)

    def gradient(ev=every):
        ax, ay, aq = gx.clone().requires_grad_(True), gy.clone().requires_grad_(True), Q.clone().requires_grad_(True)
        Ma = AD.metrics(cfg, ax, ay)
        OBJ.shock_vortex_functional(AD.rk3_march(cfg, Ma, aq, dts, ev), ax, ay, Ma, win).backward()

    march()
    gradient()
    t_fwd = C.timed(march, 1)
    t_grad = C.timed(gradient, 1)
    # every step recorded during the forward pass (no replay): 6 states per step on the device
    gradient(0)
    t_grad_tape = C.timed(lambda: gradient(0), 1)
    tape_gb = nsteps * fsp.rk3_tape(cfg, Q).numel() / 1e9
    # roofline of fsp_rhs_vjp: the oracle's operation count of one right-hand-side adjoint
    # (its forward right-hand side, the partial derivatives and the reverse sweep), per node
    with open(os.path.join(ROOT, "paper_1810_11103_gb300", "algorithmic_flops.json")) as f:
        vjp_flops = json.load(f)["adjoint"]["schemes"][SCHEME_NAMES[args.scheme]]["vjp_per_node"]
    peak, _ = C.peak("fp64")
    achieved = vjp_flops * x.size / t_rhs_vjp / 1e12
    nom = C.nominal("fp64", None)
    roof = {"bound": "alu", "kernel": "fsp_rhs_vjp (its forward right-hand side and the adjoint kernels)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "nominal_peak": nom, "frac_vs_nominal": achieved / nom, "flops_per_node": vjp_flops,
            "units_per_launch": x.size, "peak_source": "FP64 FMA probe (fsp_fma_peak) in this run"}
    return {
        "workload": f"shock_vortex512: 512x512 stretched grid, Mach 1.1 shock + vortex, {SCHEME_NAMES[args.scheme]}, "
                    f"FP64, {nsteps} RK3 steps at CFL 0.5, checkpoint every {every}",
        "rhs_ms": 1e3 * t_rhs, "rhs_vjp_ms": 1e3 * t_rhs_vjp, "rhs_vjp_over_rhs": t_rhs_vjp / t_rhs,
        "rk3_step_ms": 1e3 * t_rk3, "rk3_step_vjp_ms": 1e3 * t_rk3_vjp, "rk3_step_vjp_over_rk3_step": t_rk3_vjp / t_rk3,
        "march_forward_s": t_fwd, "march_gradient_s": t_grad, "gradient_over_forward": t_grad / t_fwd,
        "full_tape": {"march_gradient_s": t_grad_tape, "gradient_over_forward": t_grad_tape / t_fwd,
                      "tape_gb": tape_gb, "how": "every step recorded in the forward pass, no replay"},
        "roofline": roof,
    }


def _march(fsp, cfg, M, Q, dts, ws):
    for d in dts:
        fsp.rk3_step(cfg, M, Q, d, ws=ws)
    return Q


def _cfl_schedule(fsp, cfg, M, Q, tfinal, ws, cfl=0.5):
    """The time steps of an FP64 march at the CFL number to tfinal (last step clipped),
    marching Q in place: dt from fsp_cfl_dt before every step."""
    dts, t = [], 0.0
    while t < tfinal - 1e-14:
        d = min(float(fsp.cfl_dt(cfg, M, Q, cfl, ws=ws).item()), tfinal - t)
        fsp.rk3_step(cfg, M, Q, d, ws=ws)
        dts.append(d)
        t += d
    return dts


def _rho_err(a, b):
    e = (a[0] - b[0]).double()
    return {"L2": float(e.pow(2).mean().sqrt()), "Linf": float(e.abs().max())}


def measure_accuracy(args, C, full=False):
    """Final-time errors of each precision on the paper-shaped synthetic cases.
    vortex256: the 256 x 256 randomised periodic vortex over one period (t = 10, where the
    exact solution is the initial state), every scheme, CFL 0.5 (the FP64 march's steps
    replayed by the float paths): density L2 (root mean square) and Linf against the exact
    solution, and of each float path against the FP64 path.  free_stream: uniform flow
    (1, 1, 1, 1) on the same grid, max |dQ/dt| of one right-hand side and L2 of v - v0 after
    100 steps.  riemann1024 (full only): the four-quadrant problem on the partially randomised
    1024 x 1024 grid to t = 0.3, WENOIU5-1MP, float paths against FP64."""
    import numpy as np
    torch, fsp = C.torch, C.fsp
    from paper_1810_11103_gb300 import inputs as I
    dev = C.dev
    x, y, per, q = vortex_workload()
    gx, gy = torch.as_tensor(x, device=dev), torch.as_tensor(y, device=dev)
    out = {"vortex256": {}, "free_stream": {}}
    for scheme in range(4):
        res = {}
        cfg = {p: fsp.Config.from_dict(dict(scheme=scheme, precision=v, period=per)) for p, v in PRECISIONS.items()}
        M = fsp.metrics(cfg["fp64"], gx, gy)
        Q0 = torch.as_tensor(q, device=dev)
        Q64 = Q0.clone()
        dts = _cfl_schedule(fsp, cfg["fp64"], M, Q64, 10.0, fsp.workspace(cfg["fp64"], Q64))
        res["steps"] = len(dts)
        res["fp64"] = {"vs_exact": _rho_err(Q64, Q0)}
        for p in ("fp32", "mixed"):
            Qs = Q0.float().contiguous()
            _march(fsp, cfg[p], M, Qs, dts, fsp.workspace(cfg[p], Qs))
            res[p] = {"vs_exact": _rho_err(Qs, Q0), "vs_fp64": _rho_err(Qs, Q64)}
        out["vortex256"][SCHEME_NAMES[scheme]] = res
        # free stream on the same grid
        fs = {}
        qu = I.uniform_state(x.shape, 1.0, 1.0, 1.0, 1.0)
        for p, c in cfg.items():
            sdt = torch.float64 if p == "fp64" else torch.float32
            Qu = torch.as_tensor(qu, dtype=sdt, device=dev)
            ws = fsp.workspace(c, Qu)
            r = float(fsp.rhs(c, M, Qu, ws=ws).abs().max())
            d = float(fsp.cfl_dt(cfg["fp64"], M, Qu.double(), 0.5).item())
            _march(fsp, c, M, Qu, [d] * 100, ws)
            v = (Qu[2].double() / Qu[0].double() - 1.0)
            fs[p] = {"rhs_max": r, "v_L2_after_100_steps": float(v.pow(2).mean().sqrt())}
        out["free_stream"][SCHEME_NAMES[scheme]] = fs
    out["vortex256"]["how"] = ("t = 10 (one period), CFL 0.5 steps of the FP64 march replayed by the float paths; "
                               "density errors, L2 = root mean square over nodes")
    if full:
        xr, yr = I.riemann_grid(1024, 0.3, 1811)
        qr = I.riemann_quadrants(xr, yr)
        cfg = {p: fsp.Config.from_dict(dict(scheme=args.scheme, precision=v, bc=(1, 1, 1, 1)))
               for p, v in PRECISIONS.items()}
        M = fsp.metrics(cfg["fp64"], torch.as_tensor(xr, device=dev), torch.as_tensor(yr, device=dev))
        Q0 = torch.as_tensor(qr, device=dev)
        Q64 = Q0.clone()
        dts = _cfl_schedule(fsp, cfg["fp64"], M, Q64, 0.3, fsp.workspace(cfg["fp64"], Q64))
        rr = {"steps": len(dts), "scheme": SCHEME_NAMES[args.scheme]}
        for p in ("fp32", "mixed"):
            Qs = Q0.float().contiguous()
            _march(fsp, cfg[p], M, Qs, dts, fsp.workspace(cfg[p], Qs))
            e = _rho_err(Qs, Q64)
            e["Linf_rel"] = e["Linf"] / float(Q64[0].abs().max())
            rr[p] = {"vs_fp64": e}
        out["riemann1024"] = rr
    return out


def profile_run(args, prec):
    """Minimal launch sequence for a profiler: metrics, one right-hand side (line maxima,
    xi sweep, eta sweep), three launches of one direction's batched sweep alone, then one RK3
    step (the stage kernels)."""
    import numpy as np
    import torch
    from paper_1810_11103_gb300 import build as B
    B.build()
    from paper_1810_11103_gb300 import fsp
    blocks, states, free = cylinder_workload()
    cfg = fsp.Config.from_dict(dict(scheme=args.scheme, precision=PRECISIONS[prec], bc_state=np.tile(free, (4, 1))))
    bt = fsp.Batch(cfg, blocks, states)
    bt.metrics()
    for d, v in enumerate(args.profile_tiles.split(",")):
        bt.set_tile_shape(d, int(v))
    bt.rhs()
    D = [torch.empty(q.shape, dtype=torch.float32 if prec == "fp32" else torch.float64, device="cuda") for q in bt.Q]
    for _ in range(3):
        bt.flux_difference(args.profile_dir, D)
    bt.rk3_step(1e-5)   # the stage kernels: line maxima, xi, eta with the stage epilogue
    torch.cuda.synchronize()
    print(f"profile run done: {prec}, {sum(b['x'].size for b in blocks)} nodes")
    bt.close()


def profile_adjoint(args):
    """Minimal launch sequence for a profiler: three right-hand-side adjoints (each a forward
    right-hand side, then the adjoint kernels) on the 512 x 512 shock-vortex case."""
    import torch
    from paper_1810_11103_gb300 import build as B
    B.build()
    from paper_1810_11103_gb300 import fsp
    from paper_1810_11103_gb300 import inputs as I
    x, y = I.shock_vortex_grid(512)
    bc, st = I.shock_vortex_bc()
    cfg = fsp.Config.from_dict(dict(scheme=args.scheme, bc=bc, bc_state=st, eps=1e-6))
    Q = torch.as_tensor(I.shock_vortex_state(x, y), device="cuda")
    M = fsp.metrics(cfg, torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"))
    g = torch.as_tensor(I.smooth_field(x.shape, 7), device="cuda").expand(4, -1, -1).contiguous()
    Qb, Mb, ws = torch.zeros_like(Q), torch.zeros_like(M), fsp.vjp_workspace(cfg, Q)
    for _ in range(3):
        fsp.rhs_vjp(cfg, M, Q, g, Qb, Mb, ws=ws)
    torch.cuda.synchronize()
    print("profile run done: adjoint, 262144 nodes")


def measure_3d(args, C, n=128, steps=10):
    """The three-dimensional path (Sections 2.1-2.2, fsp3_*): a randomised periodic cube of n^3
    nodes (A = 0.2, seed 1810) carrying the vortex about the z axis on the free stream (1, 1, 1,
    1, 1), WENOIU5-1MP, FP64.  One step = one RK3 step (3 right-hand sides); the roofline is the
    whole right-hand side (line maxima and the three sweeps, timed together through fsp3_rhs)
    against the oracle's operation count per node.  State and metrics (290 MB) exceed L2."""
    import numpy as np
    torch, fsp = C.torch, C.fsp
    from paper_1810_11103_gb300 import inputs as I
    x, y, z, per = I.periodic_cube(n, 10.0, 0.2, seed=1810)
    q = I.vortex3(x, y, z, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0, 1.0), period=per)
    cfg = fsp.Config.from_dict(dict(scheme=2))

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=C.dev)

    blk = fsp.block3_of(dev(x), (0,) * 6, per)
    ws = fsp.workspace3(cfg, blk, C.dev)
    M = fsp.metrics3(cfg, blk, dev(x), dev(y), dev(z), ws=ws)
    Q, out = dev(q), torch.empty((5,) + x.shape, dtype=torch.float64, device=C.dev)
    dt = 1e-4
    for _ in range(max(3, args.warmup)):
        fsp.rk3_step3(cfg, blk, M, Q, dt, ws=ws)
    t = C.timed(lambda: fsp.rk3_step3(cfg, blk, M, Q, dt, ws=ws), steps)
    t_rhs = C.timed(lambda: fsp.rhs3(cfg, blk, M, Q, out=out, ws=ws), steps) / steps
    (t, t_rhs) = C.max_over_ranks(t, t_rhs)
    with open(os.path.join(ROOT, "paper_1810_11103_gb300", "algorithmic_flops.json")) as f:
        flops = json.load(f)["three_d"]["schemes"][SCHEME_NAMES[2]]["rhs_per_node"]
    nodes = n ** 3
    peak, _ = C.peak("fp64")
    achieved = flops * nodes / t_rhs / 1e12
    nominal = C.nominal("fp64", None)
    return {"workload": f"{n}^3 randomised periodic cube (A = 0.2), vortex about z, WENOIU5-1MP, FP64, TVD-RK3",
            "value": job_rhs(nodes, steps, C.world) / t / 1e6, "unit": UNIT, "ms_per_step": t / steps * 1e3,
            "roofline": {"bound": "alu", "kernel": "fsp3_rhs (line maxima + xi, eta, zeta sweeps)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "nominal_peak": nominal, "frac_vs_nominal": achieved / nominal, "flops_per_node": flops,
                         "rhs_ms": t_rhs * 1e3, "peak_source": "FP64 FMA probe (fsp_fma_peak) in this run"}}


def _r(v, d=4):
    return None if v is None else float(f"{v:.{d}g}")


def summary(args, head, others, adjoint, seventh, three_d=None):
    """Compact per-path figures: Mcell-RHS/s, ms per RK3 step, the roofline kernel's fraction of
    the measured and of the nominal FMA rate, and the per-block loop with the batching gain."""
    out = {}
    for p, r in [(args.precision, head)] + list(others.items()):
        rf = r["roofline"]
        e = {"value": _r(r["value"]), "ms_step": _r(r["ms_per_step"]), "e2e": _r(r["e2e"]["value"]),
             "kernel": rf.get("direction", "xi"), "frac": _r(rf["frac"], 3),
             "frac_nominal": _r(rf.get("frac_vs_nominal"), 3)}
        for d in ("xi", "eta"):
            if rf.get(d):
                e[d + "_ms"], e[d + "_frac"] = _r(rf[d]["kernel_ms"]), _r(rf[d]["frac"], 3)
        if rf.get("step_frac"):
            e["step_frac"] = _r(rf["step_frac"], 3)
        if p == "mixed":
            e["part"] = rf.get("part")
        if r.get("per_block"):
            e["per_block"] = _r(r["per_block"]["value"])
            e["batch_gain"] = _r(r["value"] / r["per_block"]["value"], 3)
        out["fp32_mixed" if p == "mixed" else p] = e
    if adjoint is not None:
        out["adjoint"] = {"rhs": _r(adjoint["rhs_vjp_over_rhs"], 3), "rk3": _r(adjoint["rk3_step_vjp_over_rk3_step"], 3),
                          "grad_ckpt": _r(adjoint["gradient_over_forward"], 3),
                          "grad_tape": _r(adjoint["full_tape"]["gradient_over_forward"], 3)}
        if adjoint.get("roofline"):
            out["adjoint"]["frac"] = _r(adjoint["roofline"]["frac"], 3)
    if seventh is not None:
        out["wenoiu7"] = {p: {"value": _r(seventh[p]["value"]), "frac": _r(seventh[p]["roofline"]["frac"], 3)}
                          for p in ("fp64", "fp32")}
    if three_d is not None:
        out["three_d"] = {"value": _r(three_d["value"]), "ms_step": _r(three_d["ms_per_step"]),
                          "frac": _r(three_d["roofline"]["frac"], 3)}
    return out


def profile_three_d(args):
    """Minimal launch sequence for a profiler: the three-dimensional metrics and one right-hand
    side (line maxima, xi, eta and zeta sweeps) of the bench's 128^3 cube."""
    import numpy as np
    import torch
    from paper_1810_11103_gb300 import build as B
    B.build()
    from paper_1810_11103_gb300 import fsp, inputs as I
    x, y, z, per = I.periodic_cube(128, 10.0, 0.2, seed=1810)
    q = I.vortex3(x, y, z, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0, 1.0), period=per)
    cfg = fsp.Config.from_dict(dict(scheme=2))

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")

    blk = fsp.block3_of(dev(x), (0,) * 6, per)
    ws = fsp.workspace3(cfg, blk)
    M = fsp.metrics3(cfg, blk, dev(x), dev(y), dev(z), ws=ws)
    fsp.rhs3(cfg, blk, M, dev(q), ws=ws)
    torch.cuda.synchronize()
    print("profile run done: three_d, 2097152 nodes")


def profile_probe(args):
    """Minimal launch sequence for a profiler: the FP64 FMA probe, then the FP32 one, each once
    with the launch shape of the bench's roofline peak."""
    import torch
    from paper_1810_11103_gb300 import build as B
    B.build()
    from paper_1810_11103_gb300 import fsp
    dev = torch.device("cuda", 0)
    C = Ctx(torch, fsp, None, dev, 1)
    blocks = C.sm_count() * 8
    for pipe, iters, dt in ((0, 4096, torch.float64), (1, 65536, torch.float32)):
        sink = torch.empty(blocks * 256, dtype=dt, device=dev)
        fsp.fma_peak(pipe, blocks, iters, sink)
    torch.cuda.synchronize()
    print(f"profile run done: FMA probes, {blocks} CTAs of 256 threads")


def main():
    args = parse()
    if args.profile == "adjoint":
        profile_adjoint(args)
        return
    if args.profile == "probe":
        profile_probe(args)
        return
    if args.profile == "three_d":
        profile_three_d(args)
        return
    if args.profile:
        profile_run(args, args.profile)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_1810_11103_gb300 import build as B
    B.build()
    from paper_1810_11103_gb300 import fsp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    C = Ctx(torch, fsp, dist, dev, world)

    def measure(prec, head=False):
        if args.workload == "cylinder64":
            return measure_cylinder(args, prec, C, per_block=args.per_block and prec in ("fp64", "fp32"))
        return measure_vortex(args, prec, C)

    head = measure(args.precision, head=True)
    others = {}
    if args.all_precisions:
        for p in PRECISIONS:
            if p != args.precision:
                others[p] = measure(p)
    # the adjoint covers the third- and fifth-order schemes
    adjoint = None if args.no_adjoint or args.scheme == 4 else measure_adjoint(args, C)
    accuracy = None if args.accuracy == "none" else measure_accuracy(args, C, full=args.accuracy == "full")
    seventh = None
    if args.seventh and args.scheme != 4 and args.workload == "cylinder64":
        a7 = argparse.Namespace(**dict(vars(args), scheme=4, steps=max(3, args.steps // 4)))
        seventh = {"scheme": SCHEME_NAMES[4]}
        for p in ("fp64", "fp32"):
            r = measure_cylinder(a7, p, C)
            seventh[p] = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                          "roofline": {k: r["roofline"][k] for k in ("kernel", "direction", "achieved", "peak", "unit",
                                                                   "frac", "flops_per_node", "kernel_ms")},
                          "tiles": r["tiles"]}
    three_d = measure_3d(args, C) if args.three_d and args.workload == "cylinder64" else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic", "config": workload_config(args, head["nodes"], head["nblocks"]),
            "e2e": head["e2e"],
            # per RK3 step of all blocks: 3 x (xi sweep, eta sweep) and the line maxima, one launch
            # per stage, or only the first stage's with the marching eta pass (FP64, FP32), whose
            # stages 1 and 2 take the next stage's maxima
            "gpu_launches": launches_per_step(args, head) * args.steps,
            "roofline": head["roofline"],
            "clocks": head["clocks"],
        }
        if head.get("tiles"):
            line["config"]["tiles"] = head["tiles"]
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        # the bulky tables first ...
        if accuracy is not None:
            line["accuracy"] = accuracy
        if seventh is not None:
            line["wenoiu7"] = seventh
        if three_d is not None:
            line["three_d"] = three_d
        if adjoint is not None:
            line["adjoint"] = adjoint
        for p, r in others.items():
            line["fp32_mixed" if p == "mixed" else p] = {
                "value": r["value"], "unit": UNIT, "dtype": DTYPES[p], "ms_per_step": r["ms_per_step"],
                "e2e": r["e2e"]["value"], "roofline": r["roofline"], "clocks": r["clocks"], "tiles": r.get("tiles"),
                "per_block": r.get("per_block")}
        if "per_block" in head:
            line["per_block_" + args.precision] = head["per_block"]
        # ... and a compact summary of every path last
        line["summary"] = summary(args, head, others, adjoint, seventh, three_d)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
