"""Thin Python binding of libfsp (include/fsp.h): argument marshalling only.

Every step of the computation runs in the CUDA library; torch supplies device memory
and streams.  The library must be built (``python -m paper_1810_11103_gb300.build``);
there is no fallback: a missing library or a failed call raises.

Shapes: coordinates ``x, y`` (nj, ni) float64; state ``Q`` (4, nj, ni) float64 or
float32 with unit stride along i (row stride = ld); metrics (5, nj+8, ni+8) float64.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from typing import Optional, Sequence

import torch

G = 4
FP64, FP32 = 0, 1
WENOIU3_1MP, WENOIU3_2MP, WENOIU5_1MP, WENOIU5_2MP, WENOIU7_1MP, WENOIU7_4MP = 0, 1, 2, 3, 4, 5
BC_PERIODIC, BC_TRANSMISSIVE, BC_DIRICHLET, BC_SLIPWALL, BC_FARFIELD, BC_LINK = 0, 1, 2, 3, 4, 5
FP32_MIXED = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsp.so")

_STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration", 3: "CUDA error",
           4: "non-finite value", 5: "device wait timed out", 6: "out of memory"}


class FspError(RuntimeError):
    def __init__(self, name, code):
        super().__init__(f"{name}: {_STATUS.get(code, 'unknown')} (status {code})")
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("precision", ctypes.c_int), ("interp", ctypes.c_int),
                ("ppm", ctypes.c_int), ("linear_weights", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("gamma", ctypes.c_double), ("lf_alpha", ctypes.c_double), ("eps", ctypes.c_double),
                ("bc_state", (ctypes.c_double * 4) * 4), ("weights", ctypes.c_int), ("mid_split", ctypes.c_int),
                ("scheme_alpha", ctypes.c_double)]


class _Block(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("ld", ctypes.c_longlong),
                ("period", (ctypes.c_double * 2) * 2)]


class _Block3(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("nk", ctypes.c_int), ("bc", ctypes.c_int * 6),
                ("period", (ctypes.c_double * 3) * 3)]


class _Link(ctypes.Structure):
    _fields_ = [("nbr", ctypes.c_int), ("face", ctypes.c_int), ("reversed", ctypes.c_int),
                ("offset", ctypes.c_double * 2)]


@dataclasses.dataclass
class Config:
    """Mirror of fsp_config."""
    scheme: int = WENOIU5_1MP
    precision: int = FP64
    interp: int = 0
    ppm: int = 1
    linear_weights: int = 0
    bc: Sequence[int] = (0, 0, 0, 0)
    gamma: float = 1.4
    lf_alpha: float = 1.1
    eps: float = 1e-40
    bc_state: Optional[Sequence[Sequence[float]]] = None
    period: Sequence[Sequence[float]] = ((0.0, 0.0), (0.0, 0.0))
    weights: int = 0
    mid_split: int = 0
    scheme_alpha: float = 1.0

    @classmethod
    def from_dict(cls, d):
        keys = {f.name for f in dataclasses.fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in keys})

    def _c(self):
        c = _Config()
        c.scheme, c.precision, c.interp = int(self.scheme), int(self.precision), int(self.interp)
        c.ppm, c.linear_weights = int(self.ppm), int(self.linear_weights)
        for f in range(4):
            c.bc[f] = int(self.bc[f])
        c.gamma, c.lf_alpha, c.eps = float(self.gamma), float(self.lf_alpha), float(self.eps)
        st = self.bc_state if self.bc_state is not None else [[0.0] * 4] * 4
        for f in range(4):
            for v in range(4):
                c.bc_state[f][v] = float(st[f][v])
        c.weights, c.mid_split, c.scheme_alpha = int(self.weights), int(self.mid_split), float(self.scheme_alpha)
        return c


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p


def lib():
    """Load libfsp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libfsp.so not built ({LIB_PATH}); run "
                                   "`python -m paper_1810_11103_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            C, B = ctypes.POINTER(_Config), ctypes.POINTER(_Block)
            sig = {
                "fsp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
                "fsp_metrics_elems": (ctypes.c_size_t, [B]),
                "fsp_workspace_size": (ctypes.c_int, [C, B, ctypes.POINTER(ctypes.c_size_t)]),
                "fsp_metrics": (ctypes.c_int, [C, B, _P, _P, _P, _P]),
                "fsp_line_lambda": (ctypes.c_int, [C, B, _P, _P, _P, _P, _P]),
                "fsp_rhs": (ctypes.c_int, [C, B, _P, _P, _P, _P, ctypes.c_size_t, _P]),
                "fsp_rhs_noalloc": (ctypes.c_int, [C, B, _P, _P, _P, _P]),
                "fsp_flux_difference": (ctypes.c_int, [C, B, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
                "fsp_rk3_step": (ctypes.c_int, [C, B, _P, _P, ctypes.c_double, _P, ctypes.c_size_t, _P]),
                "fsp_cfl_dt": (ctypes.c_int, [C, B, _P, _P, ctypes.c_double, _P, _P, ctypes.c_size_t, _P]),
                "fsp_norms": (ctypes.c_int, [B, ctypes.c_int, _P, _P, _P, _P]),
                "fsp_check_state": (ctypes.c_int, [C, B, _P, _P, _P]),
                "fsp_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
                "fsp_round_to_float": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P]),
                "fsp_widen_to_double": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P]),
                "fsp_reciprocal_check": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
                "fsp_vjp_workspace_size": (ctypes.c_int, [C, B, ctypes.POINTER(ctypes.c_size_t)]),
                "fsp_rhs_vjp": (ctypes.c_int, [C, B, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
                "fsp_rk3_step_vjp": (ctypes.c_int, [C, B, _P, _P, ctypes.c_double, _P, _P, _P, ctypes.c_size_t, _P]),
                "fsp_metrics_vjp": (ctypes.c_int, [C, B, _P, _P, _P, _P, _P, _P]),
                "fsp_rk3_tape_size": (ctypes.c_int, [C, B, ctypes.POINTER(ctypes.c_size_t)]),
                "fsp_rk3_step_record": (ctypes.c_int, [C, B, _P, _P, ctypes.c_double, _P, ctypes.c_size_t, _P,
                                                        ctypes.c_size_t, _P]),
                "fsp_rk3_step_vjp_tape": (ctypes.c_int, [C, B, _P, _P, ctypes.c_size_t, ctypes.c_double, _P, _P, _P,
                                                          ctypes.c_size_t, _P]),
                "fsp_batch_create": (ctypes.c_int, [C, ctypes.c_int, B, ctypes.POINTER(ctypes.c_int),
                                                    ctypes.POINTER(_Link), ctypes.POINTER(ctypes.c_void_p)]),
                "fsp_batch_bind": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                                  ctypes.POINTER(_P)]),
                "fsp_batch_metrics": (ctypes.c_int, [_P, _P]),
                "fsp_batch_rhs": (ctypes.c_int, [_P, ctypes.POINTER(_P), _P]),
                "fsp_batch_rk3_step": (ctypes.c_int, [_P, ctypes.c_double, _P]),
                "fsp_batch_rk3_step_host": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_double,
                                                           _P]),
                "fsp_batch_flux_difference": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), _P]),
                "fsp_batch_capture_graph": (ctypes.c_int, [_P, ctypes.c_double, _P]),
                "fsp_batch_tune": (ctypes.c_int, [_P, ctypes.c_char_p, _P]),
                "fsp_batch_set_tile_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
                "fsp_batch_tile_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
                "fsp_batch_destroy": (ctypes.c_int, [_P]),
                "fsp3_metrics_elems": (ctypes.c_longlong, [ctypes.POINTER(_Block3)]),
                "fsp3_workspace_size": (ctypes.c_int, [C, ctypes.POINTER(_Block3), ctypes.POINTER(ctypes.c_size_t)]),
                "fsp3_metrics": (ctypes.c_int, [C, ctypes.POINTER(_Block3), _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
                "fsp3_line_lambda": (ctypes.c_int, [C, ctypes.POINTER(_Block3), _P, _P, _P, _P]),
                "fsp3_rhs": (ctypes.c_int, [C, ctypes.POINTER(_Block3), _P, _P, _P, _P, ctypes.c_size_t, _P]),
                "fsp3_rk3_step": (ctypes.c_int, [C, ctypes.POINTER(_Block3), _P, _P, ctypes.c_double, _P,
                                                 ctypes.c_size_t, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


def _check(name, code):
    if code != 0:
        raise FspError(name, code)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dtype(cfg: Config):
    return torch.float64 if cfg.precision == FP64 else torch.float32


def block_of(cfg: Config, Q: torch.Tensor) -> _Block:
    """fsp_block of a (4, nj, ni) state tensor (unit stride along i)."""
    if Q.dim() != 3 or Q.shape[0] != 4:
        raise ValueError("state must have shape (4, nj, ni)")
    if Q.stride(2) != 1 or Q.stride(0) != Q.shape[1] * Q.stride(1):
        raise ValueError("state planes must be dense with unit stride along i")
    b = _Block()
    b.nj, b.ni, b.ld = int(Q.shape[1]), int(Q.shape[2]), int(Q.stride(1))
    for a in range(2):
        for k in range(2):
            b.period[a][k] = float(cfg.period[a][k])
    return b


def _block_shape(cfg: Config, ni: int, nj: int, ld: Optional[int] = None) -> _Block:
    b = _Block()
    b.ni, b.nj, b.ld = int(ni), int(nj), int(ni if ld is None else ld)
    for a in range(2):
        for k in range(2):
            b.period[a][k] = float(cfg.period[a][k])
    return b


def workspace_size(cfg: Config, ni: int, nj: int, ld: Optional[int] = None) -> int:
    n = ctypes.c_size_t()
    _check("fsp_workspace_size", lib().fsp_workspace_size(ctypes.byref(cfg._c()),
                                                           ctypes.byref(_block_shape(cfg, ni, nj, ld)),
                                                           ctypes.byref(n)))
    return int(n.value)


def workspace(cfg: Config, Q: torch.Tensor) -> torch.Tensor:
    b = block_of(cfg, Q)
    return torch.empty(workspace_size(cfg, b.ni, b.nj, b.ld), dtype=torch.uint8, device=Q.device)


def vjp_workspace(cfg: Config, Q: torch.Tensor) -> torch.Tensor:
    b = block_of(cfg, Q)
    n = ctypes.c_size_t()
    _check("fsp_vjp_workspace_size", lib().fsp_vjp_workspace_size(ctypes.byref(cfg._c()), ctypes.byref(b),
                                                                   ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device=Q.device)


def rhs_vjp(cfg: Config, M: torch.Tensor, Q: torch.Tensor, gbar: torch.Tensor, Qbar=None, Mbar=None, ws=None,
            stream=None):
    """(Qbar, Mbar) += the adjoint of dQ/dt = rhs(M, Q) applied to gbar (FP64)."""
    b = block_of(cfg, Q)
    Qbar = torch.zeros_like(Q) if Qbar is None else Qbar
    Mbar = torch.zeros_like(M) if Mbar is None else Mbar
    ws = vjp_workspace(cfg, Q) if ws is None else ws
    _check("fsp_rhs_vjp", lib().fsp_rhs_vjp(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q),
                                            _ptr(gbar.contiguous()), _ptr(Qbar), _ptr(Mbar), _ptr(ws), ws.numel(),
                                            _stream(stream)))
    return Qbar, Mbar


def rk3_step_vjp(cfg: Config, M: torch.Tensor, Qn: torch.Tensor, dt: float, Qbar: torch.Tensor, Mbar=None,
                 ws=None, stream=None):
    """In place: Qbar (dJ/dQ^{n+1} on entry) becomes dJ/dQ^n; Mbar += the metric adjoint."""
    b = block_of(cfg, Qn)
    ws = vjp_workspace(cfg, Qn) if ws is None else ws
    _check("fsp_rk3_step_vjp", lib().fsp_rk3_step_vjp(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Qn),
                                                      float(dt), _ptr(Qbar), _ptr(Mbar), _ptr(ws), ws.numel(),
                                                      _stream(stream)))
    return Qbar, Mbar


def rk3_tape(cfg: Config, Q: torch.Tensor) -> torch.Tensor:
    """An empty step tape for states shaped like Q (device bytes)."""
    b = block_of(cfg, Q)
    n = ctypes.c_size_t()
    _check("fsp_rk3_tape_size", lib().fsp_rk3_tape_size(ctypes.byref(cfg._c()), ctypes.byref(b), ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device=Q.device)


def rk3_step_record(cfg: Config, M: torch.Tensor, Q: torch.Tensor, dt: float, tape: torch.Tensor, ws=None,
                    stream=None) -> torch.Tensor:
    """One TVD-RK3 step in place on Q, its stages kept in tape."""
    b = block_of(cfg, Q)
    ws = workspace(cfg, Q) if ws is None else ws
    _check("fsp_rk3_step_record", lib().fsp_rk3_step_record(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q),
                                                            float(dt), _ptr(tape), tape.numel(), _ptr(ws), ws.numel(),
                                                            _stream(stream)))
    return Q


def rk3_step_vjp_tape(cfg: Config, M: torch.Tensor, tape: torch.Tensor, dt: float, Qbar: torch.Tensor, Mbar=None,
                      ws=None, stream=None):
    """In place: Qbar (dJ/dQ^{n+1} on entry) becomes dJ/dQ^n for the recorded step."""
    b = block_of(cfg, Qbar)
    ws = vjp_workspace(cfg, Qbar) if ws is None else ws
    _check("fsp_rk3_step_vjp_tape", lib().fsp_rk3_step_vjp_tape(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M),
                                                                _ptr(tape), tape.numel(), float(dt), _ptr(Qbar),
                                                                _ptr(Mbar), _ptr(ws), ws.numel(), _stream(stream)))
    return Qbar, Mbar


def metrics_vjp(cfg: Config, x: torch.Tensor, y: torch.Tensor, Mbar: torch.Tensor, xbar=None, ybar=None,
                stream=None):
    """(xbar, ybar) += the adjoint of the metrics applied to Mbar."""
    nj, ni = x.shape
    xbar = torch.zeros_like(x) if xbar is None else xbar
    ybar = torch.zeros_like(y) if ybar is None else ybar
    _check("fsp_metrics_vjp", lib().fsp_metrics_vjp(ctypes.byref(cfg._c()), ctypes.byref(_block_shape(cfg, ni, nj)),
                                                    _ptr(x.contiguous()), _ptr(y.contiguous()), _ptr(Mbar.contiguous()),
                                                    _ptr(xbar), _ptr(ybar), _stream(stream)))
    return xbar, ybar


def metrics(cfg: Config, x: torch.Tensor, y: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    nj, ni = x.shape
    x = x.contiguous()
    y = y.contiguous()
    if out is None:
        out = torch.empty((5, nj + 2 * G, ni + 2 * G), dtype=torch.float64, device=x.device)
    _check("fsp_metrics", lib().fsp_metrics(ctypes.byref(cfg._c()), ctypes.byref(_block_shape(cfg, ni, nj)),
                                            _ptr(x), _ptr(y), _ptr(out), _stream(stream)))
    return out


def line_lambda(cfg: Config, M: torch.Tensor, Q: torch.Tensor, stream=None):
    b = block_of(cfg, Q)
    lx = torch.empty(b.nj, dtype=torch.float64, device=Q.device)
    le = torch.empty(b.ni, dtype=torch.float64, device=Q.device)
    _check("fsp_line_lambda", lib().fsp_line_lambda(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M),
                                                    _ptr(Q), _ptr(lx), _ptr(le), _stream(stream)))
    return lx, le


def rhs(cfg: Config, M: torch.Tensor, Q: torch.Tensor, out=None, ws=None, stream=None) -> torch.Tensor:
    b = block_of(cfg, Q)
    if out is None:
        out = torch.empty_like(Q)
    if ws is None:
        ws = workspace(cfg, Q)
    _check("fsp_rhs", lib().fsp_rhs(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q), _ptr(out),
                                    _ptr(ws), ws.numel(), _stream(stream)))
    return out


def rhs_noalloc_status(cfg: Config, M: torch.Tensor, Q: torch.Tensor, out: torch.Tensor, stream=None) -> int:
    """fsp_rhs_noalloc: the right-hand side with the library's fixed scratch array instead of a
    workspace (for callers that cannot allocate device memory).  Returns the status code."""
    b = block_of(cfg, Q)
    return int(lib().fsp_rhs_noalloc(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q), _ptr(out),
                                     _stream(stream)))


def rhs_noalloc(cfg: Config, M: torch.Tensor, Q: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """The same as rhs() through fsp_rhs_noalloc (raises on a nonzero status)."""
    if out is None:
        out = torch.empty_like(Q)
    _check("fsp_rhs_noalloc", rhs_noalloc_status(cfg, M, Q, out, stream))
    return out


def flux_difference(cfg: Config, M: torch.Tensor, Q: torch.Tensor, lam: torch.Tensor, dir: int,
                    mode: int = 0, acc=None, out=None, stream=None) -> torch.Tensor:
    """One direction of the right-hand side (see fsp_flux_difference)."""
    b = block_of(cfg, Q)
    if out is None:
        out = torch.empty_like(Q)
    _check("fsp_flux_difference", lib().fsp_flux_difference(
        ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q), _ptr(lam), int(dir), int(mode), _ptr(acc),
        _ptr(out), _stream(stream)))
    return out


def rk3_step(cfg: Config, M: torch.Tensor, Q: torch.Tensor, dt: float, ws=None, stream=None) -> torch.Tensor:
    """One TVD-RK3 step, in place on Q."""
    b = block_of(cfg, Q)
    if ws is None:
        ws = workspace(cfg, Q)
    _check("fsp_rk3_step", lib().fsp_rk3_step(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q),
                                              float(dt), _ptr(ws), ws.numel(), _stream(stream)))
    return Q


def cfl_dt(cfg: Config, M: torch.Tensor, Q: torch.Tensor, cfl: float, out=None, ws=None, stream=None):
    b = block_of(cfg, Q)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=Q.device)
    if ws is None:
        ws = workspace(cfg, Q)
    _check("fsp_cfl_dt", lib().fsp_cfl_dt(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(M), _ptr(Q),
                                          float(cfl), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def norms(A: torch.Tensor, B: Optional[torch.Tensor] = None, out=None, stream=None) -> torch.Tensor:
    """(rms, max) of A - B per variable: tensor of 8 doubles (rms_0, max_0, ...)."""
    prec = FP64 if A.dtype == torch.float64 else FP32
    cfg = Config(precision=prec)
    b = block_of(cfg, A)
    if out is None:
        out = torch.empty(8, dtype=torch.float64, device=A.device)
    _check("fsp_norms", lib().fsp_norms(ctypes.byref(b), prec, _ptr(A), _ptr(B), _ptr(out), _stream(stream)))
    return out


def check_state(cfg: Config, Q: torch.Tensor, out=None, stream=None) -> int:
    """Index j ni + i of the first node whose state is not finite or not physical, -1 if none
    (fsp_check_state; waits for the stream).  raise_on_bad(): FspError with FSP_ERR_NONFINITE."""
    b = block_of(cfg, Q)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=Q.device)
    _check("fsp_check_state", lib().fsp_check_state(ctypes.byref(cfg._c()), ctypes.byref(b), _ptr(Q), _ptr(out),
                                                    _stream(stream)))
    return int(out.item())


def raise_on_bad(cfg: Config, Q: torch.Tensor, stream=None) -> None:
    """FspError (status 4, non-finite value) naming the first bad node, if any."""
    k = check_state(cfg, Q, stream=stream)
    if k >= 0:
        err = FspError("fsp_check_state", 4)
        err.node = (k // Q.shape[2], k % Q.shape[2])
        raise err


def round_to_float(x: torch.Tensor, stream=None):
    """(integer rounding, hardware rounding) of a float64 device tensor to float32."""
    x = x.contiguous()
    a, b = torch.empty(x.shape, dtype=torch.float32, device=x.device), torch.empty(x.shape, dtype=torch.float32,
                                                                                     device=x.device)
    _check("fsp_round_to_float", lib().fsp_round_to_float(_ptr(x), _ptr(a), _ptr(b), x.numel(), _stream(stream)))
    return a, b


def widen_to_double(x: torch.Tensor, stream=None):
    """(integer widening, hardware widening) of a float32 device tensor to float64."""
    x = x.contiguous()
    a, b = torch.empty(x.shape, dtype=torch.float64, device=x.device), torch.empty(x.shape, dtype=torch.float64,
                                                                                     device=x.device)
    _check("fsp_widen_to_double", lib().fsp_widen_to_double(_ptr(x), _ptr(a), _ptr(b), x.numel(), _stream(stream)))
    return a, b


def reciprocal_check(x: torch.Tensor, stream=None):
    """(the kernels' reciprocal, the IEEE reciprocal, the kernels' reciprocal square root, the
    IEEE 1/sqrt) of a float64 device tensor (square-root entries 0 where x <= 0)."""
    x = x.contiguous()
    out = torch.empty((4,) + tuple(x.shape), dtype=x.dtype, device=x.device)
    _check("fsp_reciprocal_check", lib().fsp_reciprocal_check(_ptr(x), _ptr(out), x.numel(), _stream(stream)))
    return tuple(out)


def fma_peak(precision: int, blocks: int, iters: int, sink: torch.Tensor, stream=None):
    _check("fsp_fma_peak", lib().fsp_fma_peak(int(precision), int(blocks), int(iters), _ptr(sink),
                                              _stream(stream)))


class Batch:
    """Many structured blocks joined by linked faces (fsp_batch_*).

    blocks: list of dicts with ``x``, ``y`` (nj, ni) arrays or tensors, ``bc`` (4 codes,
    BC_LINK for joined faces), ``links`` (4 entries: None or (nbr, face, reversed)),
    optional ``offsets`` (4 entries: None or (dx, dy)) and ``period``.  states: the
    initial (4, nj, ni) state of every block (copied to the device in the precision's
    dtype).  Device memory for coordinates, metrics and states is held here; the library
    handle holds its own scratch.  ``Qflat`` is the one device buffer behind the states
    ``Q[k]`` (views, each block padded to 128 elements), for whole-batch host copies."""

    def __init__(self, cfg: Config, blocks, states, device="cuda"):
        self.cfg = cfg
        n = len(blocks)
        dt = torch.float64 if cfg.precision == FP64 else torch.float32
        self.x = [torch.as_tensor(b["x"], dtype=torch.float64, device=device).contiguous() for b in blocks]
        self.y = [torch.as_tensor(b["y"], dtype=torch.float64, device=device).contiguous() for b in blocks]
        # every block's state in one allocation (Q[k] are views at 512-byte aligned offsets),
        # so a host round trip of the whole batch is one copy each way
        sizes = [4 * x.shape[0] * x.shape[1] for x in self.x]
        offs, tot = [], 0
        for sz in sizes:
            offs.append(tot)
            tot += (sz + 127) // 128 * 128
        self.Qflat = torch.zeros(tot, dtype=dt, device=device)
        self.Q = []
        for k, q in enumerate(states):
            nj, ni = self.x[k].shape
            v = self.Qflat[offs[k]:offs[k] + sizes[k]].view(4, nj, ni)
            v.copy_(torch.as_tensor(q, dtype=dt))
            self.Q.append(v)
        self.M = [torch.empty((5, x.shape[0] + 2 * G, x.shape[1] + 2 * G), dtype=torch.float64, device=device)
                  for x in self.x]
        blk = (_Block * n)()
        bc = (ctypes.c_int * (4 * n))()
        lk = (_Link * (4 * n))()
        for k, b in enumerate(blocks):
            nj, ni = self.x[k].shape
            blk[k].ni, blk[k].nj, blk[k].ld = ni, nj, ni
            per = b.get("period", ((0.0, 0.0), (0.0, 0.0)))
            for a in range(2):
                for c in range(2):
                    blk[k].period[a][c] = float(per[a][c])
            for f in range(4):
                bc[4 * k + f] = int(b["bc"][f])
                l = (b.get("links") or [None] * 4)[f]
                if l is not None:
                    lk[4 * k + f].nbr, lk[4 * k + f].face, lk[4 * k + f].reversed = int(l[0]), int(l[1]), int(l[2])
                o = (b.get("offsets") or [None] * 4)[f]
                if o is not None:
                    lk[4 * k + f].offset[0], lk[4 * k + f].offset[1] = float(o[0]), float(o[1])
        self._h = ctypes.c_void_p()
        _check("fsp_batch_create", lib().fsp_batch_create(ctypes.byref(cfg._c()), n, blk, bc, lk,
                                                          ctypes.byref(self._h)))
        self.n = n
        self._ptrs = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        _check("fsp_batch_bind", lib().fsp_batch_bind(self._h, self._ptrs(self.x), self._ptrs(self.y),
                                                      self._ptrs(self.M), self._ptrs(self.Q)))

    def metrics(self, stream=None):
        _check("fsp_batch_metrics", lib().fsp_batch_metrics(self._h, _stream(stream)))
        return self.M

    def rhs(self, out=None, stream=None):
        out = [torch.empty_like(q) for q in self.Q] if out is None else out
        _check("fsp_batch_rhs", lib().fsp_batch_rhs(self._h, self._ptrs(out), _stream(stream)))
        return out

    def flux_difference(self, dir: int, out, stream=None):
        """One direction of every block into out[b] (after a rhs() call on this handle)."""
        _check("fsp_batch_flux_difference", lib().fsp_batch_flux_difference(self._h, int(dir), self._ptrs(out),
                                                                            _stream(stream)))
        return out

    def rk3_step(self, dt: float, stream=None):
        _check("fsp_batch_rk3_step", lib().fsp_batch_rk3_step(self._h, float(dt), _stream(stream)))
        return self.Q

    def rk3_step_host(self, dt: float, host_in: torch.Tensor, host_out: torch.Tensor, stream=None):
        """One step from and to host memory in one library call (fsp_batch_rk3_step_host):
        host_in and host_out are CPU tensors laid out like Qflat (pinned for asynchronous
        copies); host_out holds the new states once the stream has completed."""
        for t in (host_in, host_out):
            if t.device.type != "cpu" or t.dtype != self.Qflat.dtype or t.numel() != self.Qflat.numel() \
                    or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors shaped and typed like Qflat")
        key = (host_in.data_ptr(), host_out.data_ptr())
        if getattr(self, "_host_key", None) != key:       # the pointer tables of the last pair
            offs = [q.data_ptr() - self.Qflat.data_ptr() for q in self.Q]
            self._host_tabs = tuple((ctypes.c_void_p * self.n)(*[p + o for o in offs]) for p in key)
            self._host_key = key
        pin, pout = self._host_tabs
        _check("fsp_batch_rk3_step_host", lib().fsp_batch_rk3_step_host(self._h, pin, pout, float(dt),
                                                                        _stream(stream)))
        return host_out

    def capture_graph(self, dt: float, stream=None):
        _check("fsp_batch_capture_graph", lib().fsp_batch_capture_graph(self._h, float(dt), _stream(stream)))

    def tune(self, table_path: Optional[str] = None, stream=None):
        """Pick the fastest tile shape of each direction (fsp_batch_tune); returns the
        (variant, lines, output nodes) of the xi and eta tiles."""
        path = None if table_path is None else os.fsencode(table_path)
        _check("fsp_batch_tune", lib().fsp_batch_tune(self._h, path, _stream(stream)))
        return self.tile_shape(0), self.tile_shape(1)

    def set_tile_shape(self, dir: int, variant: int):
        _check("fsp_batch_set_tile_shape", lib().fsp_batch_set_tile_shape(self._h, int(dir), int(variant)))

    def tile_shape(self, dir: int):
        v, nl, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check("fsp_batch_tile_shape", lib().fsp_batch_tile_shape(self._h, int(dir), ctypes.byref(v), ctypes.byref(nl),
                                                                  ctypes.byref(t)))
        return v.value, nl.value, t.value

    def close(self):
        if getattr(self, "_h", None):
            lib().fsp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- three dimensions (fsp3_*): state (5, nk, nj, ni), coordinates (nk, nj, ni), FP64 ----------
def block3_of(Q: torch.Tensor, bc=(0, 0, 0, 0, 0, 0), period=((0.0,) * 3,) * 3) -> _Block3:
    """The fsp3_block of a state or coordinate tensor whose last three extents are (nk, nj, ni)."""
    nk, nj, ni = Q.shape[-3:]
    b = _Block3()
    b.ni, b.nj, b.nk = int(ni), int(nj), int(nk)
    for f in range(6):
        b.bc[f] = int(bc[f])
    for a in range(3):
        for c in range(3):
            b.period[a][c] = float(period[a][c])
    return b


def workspace3(cfg: Config, blk: _Block3, device="cuda") -> torch.Tensor:
    n = ctypes.c_size_t()
    _check("fsp3_workspace_size", lib().fsp3_workspace_size(ctypes.byref(cfg._c()), ctypes.byref(blk), ctypes.byref(n)))
    return torch.empty(int(n.value), dtype=torch.uint8, device=device)


def metrics3(cfg: Config, blk: _Block3, x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, out=None, ws=None,
             stream=None) -> torch.Tensor:
    out = torch.empty((10, blk.nk + 2 * G, blk.nj + 2 * G, blk.ni + 2 * G), dtype=torch.float64,
                      device=x.device) if out is None else out
    ws = workspace3(cfg, blk, x.device) if ws is None else ws
    _check("fsp3_metrics", lib().fsp3_metrics(ctypes.byref(cfg._c()), ctypes.byref(blk), _ptr(x.contiguous()),
                                              _ptr(y.contiguous()), _ptr(z.contiguous()), _ptr(out), _ptr(ws),
                                              ws.numel(), _stream(stream)))
    return out


def line_lambda3(cfg: Config, blk: _Block3, M: torch.Tensor, Q: torch.Tensor, stream=None):
    """The xi, eta and zeta line maxima (without lf_alpha): shapes (nk, nj), (nk, ni), (nj, ni)."""
    n = blk.nj * blk.nk + blk.ni * blk.nk + blk.ni * blk.nj
    lam = torch.empty(n, dtype=torch.float64, device=Q.device)
    _check("fsp3_line_lambda", lib().fsp3_line_lambda(ctypes.byref(cfg._c()), ctypes.byref(blk), _ptr(M), _ptr(Q),
                                                      _ptr(lam), _stream(stream)))
    a, b = blk.nj * blk.nk, blk.nj * blk.nk + blk.ni * blk.nk
    return (lam[:a].view(blk.nk, blk.nj), lam[a:b].view(blk.nk, blk.ni), lam[b:].view(blk.nj, blk.ni))


def rhs3(cfg: Config, blk: _Block3, M: torch.Tensor, Q: torch.Tensor, out=None, ws=None, stream=None):
    out = torch.empty_like(Q) if out is None else out
    ws = workspace3(cfg, blk, Q.device) if ws is None else ws
    _check("fsp3_rhs", lib().fsp3_rhs(ctypes.byref(cfg._c()), ctypes.byref(blk), _ptr(M), _ptr(Q), _ptr(out),
                                      _ptr(ws), ws.numel(), _stream(stream)))
    return out


def rk3_step3(cfg: Config, blk: _Block3, M: torch.Tensor, Q: torch.Tensor, dt: float, ws=None, stream=None):
    ws = workspace3(cfg, blk, Q.device) if ws is None else ws
    _check("fsp3_rk3_step", lib().fsp3_rk3_step(ctypes.byref(cfg._c()), ctypes.byref(blk), _ptr(M), _ptr(Q),
                                                float(dt), _ptr(ws), ws.numel(), _stream(stream)))
    return Q
