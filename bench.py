#!/usr/bin/env python
"""Benchmark of the WENOIU free-stream-preserving Euler right-hand side on GB300.

One step = one TVD-RK3 step (three right-hand sides: per-line spectral radius, xi sweep,
eta sweep fused with the stage update) over the whole synthetic workload, through the C
ABI of libfsp.  Metric: Mcell-RHS/s = nodes x right-hand sides / second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(n):
    """The periodic vortex case: n x n nodes on [0, 10)^2, every node randomised by up to
    +-0.2 h (seed 1810), vortex of strength 5 on the free stream (1, 1, 1, 1)."""
    from paper_1810_11103_gb300 import inputs as I
    x, y, per = I.periodic_square(n, 10.0, 0.2, seed=1810)
    q = I.isentropic_vortex(x, y, (5.0, 5.0), strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=(10.0, 10.0))
    return x, y, per, q


def config_of(args, per):
    return dict(scheme=args.scheme, precision=0, interp=0, ppm=1, linear_weights=0, bc=(0, 0, 0, 0),
                gamma=1.4, lf_alpha=1.1, eps=1e-40, period=per)


def workload_config(args):
    return {"workload": f"periodic isentropic vortex {args.n}x{args.n}, randomised grid +-0.2h, "
                        f"{SCHEME_NAMES[args.scheme]}, TVD-RK3",
            "ni": args.n, "nj": args.n, "scheme": SCHEME_NAMES[args.scheme], "precision": "fp64",
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

    x, y, per, q = workload(args.n)
    cfgd = config_of(args, per)
    cfg = fsp.Config.from_dict(cfgd)
    stream = torch.cuda.current_stream()
    X, Y = torch.as_tensor(x, device=dev), torch.as_tensor(y, device=dev)
    M = fsp.metrics(cfg, X, Y)
    Q0 = torch.as_tensor(q, device=dev)
    Q = Q0.clone()
    ws = fsp.workspace(cfg, Q)
    dt = float(fsp.cfl_dt(cfg, M, Q, 0.5, ws=ws).item())
    nodes = args.n * args.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region ----
    for _ in range(args.warmup):
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
        ev[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    launches = 9 * args.steps     # per RK3 step: 3 x (line maxima, xi sweep, eta sweep)

    # ---- end to end through the API with host buffers ----
    Qh = torch.as_tensor(q).pin_memory()
    Qout = torch.empty_like(Qh).pin_memory()
    for _ in range(2):
        Q.copy_(Qh, non_blocking=True)
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
        Qout.copy_(Q, non_blocking=True)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        Q.copy_(Qh, non_blocking=True)
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
        Qout.copy_(Q, non_blocking=True)
        ev2[k][1].record(stream)
    barrier()
    t_e2e = sum(a.elapsed_time(b) for a, b in ev2) / 1e3
    state_bytes = Q.numel() * Q.element_size()

    # ---- the dominant kernel alone: the xi sweep (fsp_flux_difference, direction 0) ----
    lx, le = fsp.line_lambda(cfg, M, Q)
    D = torch.empty_like(Q)
    for _ in range(3):
        fsp.flux_difference(cfg, M, Q, lx, 0, 0, out=D)
    ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    barrier()
    for a, b in ev3:
        flush.zero_()
        a.record(stream)
        fsp.flux_difference(cfg, M, Q, lx, 0, 0, out=D)
        b.record(stream)
    barrier()
    t_k = sum(a.elapsed_time(b) for a, b in ev3) / 1e3 / len(ev3)

    # ---- ALU roof: FP64 FMA probe at the same clocks ----
    blocks, iters = 152 * 8, 4096
    sink = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    fsp.fma_peak(0, blocks, iters, sink)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    fsp.fma_peak(0, blocks, iters, sink)
    e1.record(stream)
    barrier()
    p64 = 2.0 * 8 * iters * blocks * 256 / (e0.elapsed_time(e1) / 1e3) / 1e12

    if world > 1:
        t = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, t_e2e = float(t[0]), float(t[1])
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    with open(os.path.join(ROOT, "paper_1810_11103_gb300", "algorithmic_flops.json")) as f:
        flops = json.load(f)["schemes"][SCHEME_NAMES[args.scheme]]
    achieved = flops["sweep_xi_per_node"] * nodes / t_k / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        if tr.get("source_hash") == source_hash() and tr.get("n") == args.n and tr.get("scheme") == args.scheme:
            traffic = tr.get("bytes_per_launch")
    rhs_total = nodes * 3 * args.steps * world
    line = {
        "metric": METRIC, "value": rhs_total / t_dev / 1e6, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args),
        "e2e": {"value": rhs_total / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "sweep_kernel xi (fsp_flux_difference dir 0)",
                     "achieved": achieved, "peak": p64, "unit": "TFLOP/s", "frac": achieved / p64,
                     "traffic": traffic, "peak_source": "FP64 FMA probe (fsp_fma_peak) in this run",
                     "flops_per_node": flops["sweep_xi_per_node"], "kernel_ms": 1e3 * t_k},
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
