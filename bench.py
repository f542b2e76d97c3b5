#!/usr/bin/env python
"""Benchmark of the WENOIU free-stream-preserving Euler right-hand side on GB300.

One step = one TVD-RK3 step (three right-hand sides: per-line spectral radius, xi sweep,
eta sweep fused with the stage update) over the whole synthetic workload, through the C
ABI of libfsp.  Metric: Mcell-RHS/s = nodes x right-hand sides / second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--precision fp64|fp32|mixed] [--no-all-precisions]

The headline `value` is the FP64 path; the FP32 and mixed FP32/FP64 paths of the same
workload are reported beside it ("fp32", "fp32_mixed"), each with its own roofline.

Under torchrun every rank runs the same workload on its own GPU (independent problems,
weak scaling, no data-path collective); rank 0 prints one JSON line.
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
SCHEME_NAMES = ["WENOIU3-1MP", "WENOIU3-2MP", "WENOIU5-1MP", "WENOIU5-2MP"]
L2_FLUSH_BYTES = 256 << 20   # larger than the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--scheme", type=int, default=2)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--all-precisions", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure the other two precisions and report them beside the headline")
    return ap.parse_args()


def workload(n):
    """The periodic vortex case: n x n nodes on [0, 10)^2, every node randomised by up to
    +-0.2 h (seed 1810), vortex of strength 5 on the free stream (1, 1, 1, 1)."""
    from paper_1810_11103_gb300 import inputs as I
    x, y, per = I.periodic_square(n, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    return x, y, per, q


PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}
DTYPES = {"fp64": "f64", "fp32": "f32", "mixed": "f32+f64"}


def config_of(args, per):
    return dict(scheme=args.scheme, precision=PRECISIONS[getattr(args, "precision", "fp64")], interp=0, ppm=1, linear_weights=0, bc=(0, 0, 0, 0),
                gamma=1.4, lf_alpha=1.1, eps=1e-40, period=per)


def workload_config(args):
    return {"workload": f"periodic isentropic vortex {args.n}x{args.n}, randomised grid +-0.2h, "
                        f"{SCHEME_NAMES[args.scheme]}, TVD-RK3",
            "ni": args.n, "nj": args.n, "scheme": SCHEME_NAMES[args.scheme], "precision": args.precision,
            "step": "one RK3 step = 3 right-hand sides",
            "l2": "flushed between timed steps (256 MiB write outside the events)"}


def source_hash():
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_1810_11103_gb300", "csrc")
    for f in sorted(os.listdir(src)):
        with open(os.path.join(src, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


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


def cpu_baseline(args, seconds=12.0):
    """The oracle, as it stands, on one host core: right-hand sides of the full workload."""
    import oracle as O
    x, y, per, q = workload(args.n)
    cfg = config_of(args, per)
    M = O.metrics(cfg, x, y)
    t0 = time.perf_counter()
    k = 0
    while True:
        O.rhs(cfg, M, q)
        k += 1
        t = time.perf_counter() - t0
        if t > seconds:
            break
    return {"value": x.size * k / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k} right-hand sides of the {args.n}x{args.n} workload (oracle, one thread)"}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle as O
    O.build()
    x, y, per, q = workload(args.n)
    cfg = config_of(args, per)
    M = O.metrics(cfg, x, y)
    for _ in range(args.warmup):
        O.rhs(cfg, M, q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rhs(cfg, M, q)
    t = time.perf_counter() - t0
    value = x.size * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(workload_config(args),
                                                 step="one right-hand side (oracle, one host thread)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} right-hand sides of the {args.n}x{args.n} workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(args, prec, dev, world, rank, torch, fsp, dist):
    """Time the RK3 step (device-resident and end to end) and the dominant kernel for one
    precision of the workload; returns a dict."""
    x, y, per, q = workload(args.n)
    cfgd = dict(config_of(args, per), precision=PRECISIONS[prec])
    cfg = fsp.Config.from_dict(cfgd)
    stream = torch.cuda.current_stream()
    X, Y = torch.as_tensor(x, device=dev), torch.as_tensor(y, device=dev)
    M = fsp.metrics(cfg, X, Y)
    sdt = torch.float64 if prec == "fp64" else torch.float32
    Q = torch.as_tensor(q, dtype=sdt, device=dev)
    ws = fsp.workspace(cfg, Q)
    dt = float(fsp.cfl_dt(cfg, M, Q, 0.5, ws=ws).item())
    nodes = args.n * args.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(body, reps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        barrier()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            body()
            b.record(stream)
        barrier()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    for _ in range(args.warmup):
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    t_dev = timed(lambda: fsp.rk3_step(cfg, M, Q, dt, ws=ws), args.steps)
    clk = clocks.stop()

    # end to end through the API: pinned host state in, RK3 step, state back to the host
    Qh = torch.as_tensor(q, dtype=sdt).pin_memory()
    Qout = torch.empty_like(Qh).pin_memory()

    def e2e():
        Q.copy_(Qh, non_blocking=True)
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
        Qout.copy_(Q, non_blocking=True)
    for _ in range(2):
        e2e()
    t_e2e = timed(e2e, args.steps)

    # the dominant kernel alone: the xi sweep (fsp_flux_difference, direction 0)
    lx, le = fsp.line_lambda(cfg, M, Q)
    D = torch.empty(Q.shape, dtype=torch.float32 if prec == "fp32" else torch.float64, device=dev)
    for _ in range(3):
        fsp.flux_difference(cfg, M, Q, lx, 0, 0, out=D)
    t_k = timed(lambda: fsp.flux_difference(cfg, M, Q, lx, 0, 0, out=D), 20) / 20

    # ALU roof: FMA probe of the precision that bounds the kernel
    pipe = 0 if prec == "fp64" else 1
    blocks, iters = 152 * 8, 4096 if pipe == 0 else 65536
    sink = torch.empty(blocks * 256, dtype=torch.float64 if pipe == 0 else torch.float32, device=dev)
    fsp.fma_peak(pipe, blocks, iters, sink)
    t_p = timed(lambda: fsp.fma_peak(pipe, blocks, iters, sink), 3) / 3
    peak = 2.0 * 8 * iters * blocks * 256 / t_p / 1e12

    if world > 1:
        t = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, t_e2e = float(t[0]), float(t[1])
    with open(os.path.join(ROOT, "paper_1810_11103_gb300", "algorithmic_flops.json")) as f:
        flops = json.load(f)["schemes"][SCHEME_NAMES[args.scheme]]
    achieved = flops["sweep_xi_per_node"] * nodes / t_k / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        if (tr.get("source_hash") == source_hash() and tr.get("n") == args.n and tr.get("scheme") == args.scheme
                and tr.get("precision", "fp64") == prec):
            traffic = tr.get("bytes_per_launch")
    rhs_total = nodes * 3 * args.steps * world
    state_bytes = Q.numel() * Q.element_size()
    return {
        "value": rhs_total / t_dev / 1e6, "ms_per_step": 1e3 * t_dev / args.steps,
        "e2e": {"value": rhs_total / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "roofline": {"bound": "alu", "kernel": "sweep_kernel xi (fsp_flux_difference dir 0)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "peak_source": ("FP64" if pipe == 0 else "FP32") + " FMA probe (fsp_fma_peak) in this run",
                     "flops_per_node": flops["sweep_xi_per_node"], "kernel_ms": 1e3 * t_k},
        "clocks": clk,
    }


def main():
    args = parse()
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

    head = measure(args, args.precision, dev, world, rank, torch, fsp, dist)
    others = {}
    if args.all_precisions:
        for p in ("fp64", "fp32", "mixed"):
            if p != args.precision:
                others[p] = measure(args, p, dev, world, rank, torch, fsp, dist)
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic", "config": workload_config(args),
            "e2e": head["e2e"],
            "gpu_launches": 9 * args.steps,   # per RK3 step: 3 x (line maxima, xi sweep, eta sweep)
            "roofline": head["roofline"],
            "clocks": head["clocks"],
        }
        for p, r in others.items():
            line["fp32_mixed" if p == "mixed" else p] = {
                "value": r["value"], "unit": UNIT, "dtype": DTYPES[p], "ms_per_step": r["ms_per_step"],
                "e2e": r["e2e"]["value"], "roofline": r["roofline"], "clocks": r["clocks"]}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
