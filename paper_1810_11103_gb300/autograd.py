"""PyTorch autograd wrappers over the library's discrete adjoint.

FspMetrics  (x, y)     -> metrics        backward: fsp_metrics_vjp
FspRHS      (M, Q)     -> dQ/dt          backward: fsp_rhs_vjp
FspRK3      (M, Q0)    -> Q after the given TVD-RK3 steps (Section 6, Shu-Osher form)
                                         backward: fsp_rk3_step_vjp, step by step in reverse,
                                         recomputing each segment's states from checkpoints

Every backward runs in the library's kernels (FP64); these classes only order the calls
and hold the tensors.  The time steps of a march are inputs, not functions of the state:
a march whose steps come from the CFL condition takes them from ``cfl_schedule`` and the
gradient holds them fixed.
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import fsp


def _need_fp64(cfg: fsp.Config):
    if cfg.precision != 0:
        raise ValueError("the adjoint is FP64 only (precision 0)")


class FspMetrics(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cfg: fsp.Config, x: torch.Tensor, y: torch.Tensor):
        ctx.cfg = cfg
        ctx.save_for_backward(x, y)
        return fsp.metrics(cfg, x.contiguous(), y.contiguous())

    @staticmethod
    def backward(ctx, Mbar):
        x, y = ctx.saved_tensors
        xb, yb = fsp.metrics_vjp(ctx.cfg, x.contiguous(), y.contiguous(), Mbar.contiguous())
        return None, xb, yb


class FspRHS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cfg: fsp.Config, M: torch.Tensor, Q: torch.Tensor):
        _need_fp64(cfg)
        ctx.cfg = cfg
        M, Q = M.contiguous(), Q.contiguous()
        ctx.save_for_backward(M, Q)
        return fsp.rhs(cfg, M, Q)

    @staticmethod
    def backward(ctx, gbar):
        M, Q = ctx.saved_tensors
        Qb, Mb = fsp.rhs_vjp(ctx.cfg, M, Q, gbar.contiguous())
        return None, Mb, Qb


class FspRK3(torch.autograd.Function):
    """Q0 advanced by len(dts) TVD-RK3 steps.  Every ``every``-th state is kept; the
    backward pass replays one segment at a time from its checkpoint, recording each step's
    stages (fsp_rk3_step_record), and runs the recorded steps' adjoints in reverse
    (fsp_rk3_step_vjp_tape), so memory holds about len(dts)/every states and every step
    tapes.  every <= 0 records every step during the forward pass and replays nothing."""

    @staticmethod
    def forward(ctx, cfg: fsp.Config, M: torch.Tensor, Q0: torch.Tensor, dts: Sequence[float], every: int):
        _need_fp64(cfg)
        ctx.cfg, ctx.dts = cfg, tuple(float(d) for d in dts)
        n = len(ctx.dts)
        ctx.every = max(n, 1) if every <= 0 else int(every)
        ctx.taped = every <= 0
        M = M.contiguous()
        Q = Q0.detach().clone(memory_format=torch.contiguous_format)
        ws = fsp.workspace(cfg, Q)
        keep = []
        for k, dt in enumerate(ctx.dts):
            if ctx.taped:
                keep.append(fsp.rk3_tape(cfg, Q))
                fsp.rk3_step_record(cfg, M, Q, dt, keep[-1], ws=ws)
                continue
            if k % ctx.every == 0:
                keep.append(Q.clone())
            fsp.rk3_step(cfg, M, Q, dt, ws=ws)
        ctx.save_for_backward(M, *keep)
        return Q

    @staticmethod
    def backward(ctx, QNbar):
        M, *keep = ctx.saved_tensors
        cfg, dts = ctx.cfg, ctx.dts
        n = len(dts)
        Qb = QNbar.detach().clone(memory_format=torch.contiguous_format)
        Mb = torch.zeros_like(M)
        if n == 0:
            return None, Mb, Qb, None, None
        vws = fsp.vjp_workspace(cfg, Qb)
        if ctx.taped:
            for k in range(n - 1, -1, -1):
                fsp.rk3_step_vjp_tape(cfg, M, keep[k], dts[k], Qb, Mb, ws=vws)
            return None, Mb, Qb, None, None
        ws = fsp.workspace(cfg, Qb)
        seg = ctx.every
        tapes = [fsp.rk3_tape(cfg, Qb) for _ in range(min(seg, n))]
        for s in range((n - 1) // seg, -1, -1):
            lo, hi = s * seg, min(n, (s + 1) * seg)
            Q = keep[s].clone()
            for k in range(lo, hi):               # replay the segment, recording each step
                fsp.rk3_step_record(cfg, M, Q, dts[k], tapes[k - lo], ws=ws)
            for k in range(hi - 1, lo - 1, -1):
                fsp.rk3_step_vjp_tape(cfg, M, tapes[k - lo], dts[k], Qb, Mb, ws=vws)
        return None, Mb, Qb, None, None


def metrics(cfg: fsp.Config, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    return FspMetrics.apply(cfg, x, y)


def rhs(cfg: fsp.Config, M: torch.Tensor, Q: torch.Tensor) -> torch.Tensor:
    return FspRHS.apply(cfg, M, Q)


def rk3_march(cfg: fsp.Config, M: torch.Tensor, Q0: torch.Tensor, dts: Sequence[float],
              every: int = 14) -> torch.Tensor:
    return FspRK3.apply(cfg, M, Q0, tuple(dts), every)


@torch.no_grad()
def cfl_schedule(cfg: fsp.Config, M: torch.Tensor, Q0: torch.Tensor, nsteps: int, cfl: float):
    """The time steps of an nsteps march at the given CFL number (each from fsp_cfl_dt on
    the state it starts from), and the final state."""
    Q = Q0.detach().clone(memory_format=torch.contiguous_format)
    ws = fsp.workspace(cfg, Q)
    dts = []
    for _ in range(nsteps):
        dt = float(fsp.cfl_dt(cfg, M, Q, cfl, ws=ws).item())
        dts.append(dt)
        fsp.rk3_step(cfg, M, Q, dt, ws=ws)
    return dts, Q
