"""ctypes front end of the CPU oracle (test infrastructure only).

Builds ``_build/libfsp_oracle.so`` from ``fsp_oracle.cpp`` with g++ (``-O2
-ffp-contract=off``, no OpenMP: the oracle runs on one core) and exposes numpy-level
functions.  The configuration is a plain dict with the keys

    scheme          0..5 = WENOIU3-1MP, WENOIU3-2MP, WENOIU5-1MP, WENOIU5-2MP, WENOIU7-1MP,
                    WENOIU7-4MP (the last on periodic grids only)
    interp          0 = order-matched Lagrange midpoint interpolation, 1 = 2-point average
    ppm             1 = piecewise-polynomial mapping of the weights (Eqs. 3.15/3.23)
    linear_weights  1 = omega_k = C_k (linear interpolation)
    bc              4 face codes (i-min, i-max, j-min, j-max): 0 periodic, 1 transmissive,
                    2 Dirichlet, 3 slip wall, 4 far field
    bc_state        4 x 4 conservative states used by Dirichlet / far-field faces
    gamma, lf_alpha, eps
    period          ((dx, dy) per wrap in i, (dx, dy) per wrap in j)

Arrays: coordinates ``x, y`` are (nj, ni); the state ``Q`` is (4, nj, ni); metrics are
(5, nj+8, ni+8) planes (xi_x^, xi_y^, eta_x^, eta_y^, J^-1) with 4 ghost layers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "lib", "metrics", "metrics_jvp", "line_lambda", "rhs", "rhs_jvp", "rk3", "rk3_jvp",
    "cfl_dt", "count_flops", "count_mid_interp", "count_char_dir", "count_flops_parts", "fsp_residual", "weno", "ppm", "smoothness", "eig",
    "scheme_table", "advect1d", "advect1d_dt", "smoothness4", "riemann_exact", "long_double_digits", "G",
    "mb_metrics", "mb_rhs", "mb_rk3", "rhs_vjp", "rk3_vjp", "metrics_vjp", "count_vjp_flops",
    "advect1d_opts", "weno_z", "split_flux",
    "metrics3", "rhs3", "rk3_3", "lambda3", "count_flops3", "eig3", "fsp_residual3",
]

G = 4
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsp_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libfsp_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2 -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # FSP_ORACLE_LIB: a separately built copy of the oracle (the mutation tests build
            # copies with a planted mistake and run the pins against them)
            L = ctypes.CDLL(os.environ.get("FSP_ORACLE_LIB") or build())
            sig = {
                "orc_metrics": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]),
                "orc_metrics_jvp": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D]),
                "orc_lambda": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]),
                "orc_rhs": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D]),
                "orc_rhs_jvp": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D]),
                "orc_rk3": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int]),
                "orc_rk3_jvp": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                               ctypes.c_double, ctypes.c_int]),
                "orc_cfl_dt": (ctypes.c_double, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double]),
                "orc_count_flops": (ctypes.c_longlong, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D]),
                "orc_count_mid_interp": (ctypes.c_longlong, [ctypes.c_int, ctypes.c_int]),
                "orc_count_char_dir": (ctypes.c_longlong, []),
                "orc_count_flops_parts": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D,
                                                         ctypes.POINTER(ctypes.c_longlong)]),
                "orc_fsp_residual": (ctypes.c_double, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                                       ctypes.c_int]),
                "orc_weno": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]),
                "orc_ppm": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double]),
                "orc_smoothness": (None, [_D, _D]),
                "orc_eig": (None, [ctypes.c_double, _D, ctypes.c_double, ctypes.c_double, _D, _D]),
                "orc_scheme_table": (None, [ctypes.c_int, ctypes.c_double, _D]),
                "orc_advect1d": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]),
                "orc_advect1d_dt": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]),
                "orc_smoothness4": (None, [_D, _D]),
                "orc_advect1d_opts": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_int, _D]),
                "orc_weno_z": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, _D]),
                "orc_split_flux": (ctypes.c_int, [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  _D, _D, _D]),
                "orc_riemann_exact": (ctypes.c_int, [ctypes.c_double, _D, _D, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_int, _D, _D]),
                "orc_long_double_digits": (ctypes.c_int, []),
                "orc_rhs_vjp": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]),
                "orc_rk3_vjp": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, _D, _D]),
                "orc_metrics_vjp": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D]),
                "orc_count_vjp_flops": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, _D, _D,
                                                       ctypes.POINTER(ctypes.c_longlong)]),
                "orc_mb_metrics": (ctypes.c_int, [_I, _D, ctypes.c_int, _I, _I, _I, _D, _D, _D, _D, _D]),
                "orc_mb_rhs": (ctypes.c_int, [_I, _D, ctypes.c_int, _I, _I, _I, _D, _D, _D]),
                "orc_mb_rk3": (ctypes.c_int, [_I, _D, ctypes.c_int, _I, _I, _I, _D, _D, ctypes.c_double,
                                              ctypes.c_int]),
                "orc3_metrics_len": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc3_metrics": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]),
                "orc3_rhs": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]),
                "orc3_rk3": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                            ctypes.c_double, ctypes.c_int]),
                "orc3_lambda": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               _D, _D, _D]),
                "orc3_count_flops": (ctypes.c_int, [_I, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                                    ctypes.POINTER(ctypes.c_longlong)]),
                "orc3_eig": (None, [ctypes.c_double, _D, _D, _D, _D]),
                "orc3_fsp_residual": (ctypes.c_double, [_I, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                                        _D, _D, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _params(cfg):
    """ip = (scheme, interp, ppm, linear_weights, bc[4], weights, mid_split); dp = (gamma,
    lf_alpha, eps, bc_state[4][4], scheme_alpha)."""
    alpha = float(cfg.get("scheme_alpha", 1.0))
    if alpha != 1.0 and cfg.get("scheme", 2) in (1, 3, 5):
        raise ValueError("oracle: the two-midpoint schemes have no free parameter")
    ip = np.array([cfg.get("scheme", 2), cfg.get("interp", 0), cfg.get("ppm", 1),
                   cfg.get("linear_weights", 0)] + list(cfg.get("bc", (0, 0, 0, 0)))
                  + [cfg.get("weights", 0), cfg.get("mid_split", 0)], dtype=np.int32)
    st = np.zeros((4, 4)) if cfg.get("bc_state") is None else np.asarray(cfg["bc_state"], dtype=np.float64)
    dp = np.concatenate([[cfg.get("gamma", 1.4), cfg.get("lf_alpha", 1.1), cfg.get("eps", 1e-40)],
                         st.reshape(16), [alpha]]).astype(np.float64)
    per = np.asarray(cfg.get("period", ((0.0, 0.0), (0.0, 0.0))), dtype=np.float64).reshape(4)
    return ip, dp, per


def _ck(rc, name):
    if rc != 0:
        raise ValueError(f"oracle {name}: invalid arguments (code {rc})")


def metrics(cfg, x, y):
    x, y = _f64(x), _f64(y)
    nj, ni = x.shape
    ip, dp, per = _params(cfg)
    M = np.empty((5, nj + 2 * G, ni + 2 * G))
    _ck(lib().orc_metrics(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(per), _dp(x), _dp(y), _dp(M)), "metrics")
    return M


def metrics_jvp(cfg, x, y, dx, dy):
    x, y, dx, dy = _f64(x), _f64(y), _f64(dx), _f64(dy)
    nj, ni = x.shape
    ip, dp, per = _params(cfg)
    M = np.empty((5, nj + 2 * G, ni + 2 * G))
    dM = np.empty_like(M)
    _ck(lib().orc_metrics_jvp(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(per), _dp(x), _dp(y), _dp(dx), _dp(dy),
                              _dp(M), _dp(dM)), "metrics_jvp")
    return M, dM


def line_lambda(cfg, M, Q):
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    lx, le = np.empty(nj), np.empty(ni)
    _ck(lib().orc_lambda(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), _dp(lx), _dp(le)), "lambda")
    return lx, le


def rhs(cfg, M, Q):
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    R = np.empty_like(Q)
    _ck(lib().orc_rhs(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), _dp(R)), "rhs")
    return R


def rhs_jvp(cfg, M, Q, dM=None, dQ=None):
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    dM = np.zeros_like(M) if dM is None else _f64(dM)
    dQ = np.zeros_like(Q) if dQ is None else _f64(dQ)
    R, dR = np.empty_like(Q), np.empty_like(Q)
    _ck(lib().orc_rhs_jvp(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(dM), _dp(Q), _dp(dQ),
                          _dp(R), _dp(dR)), "rhs_jvp")
    return R, dR


def rk3(cfg, M, Q, dt, nsteps=1):
    M = _f64(M)
    Q = np.array(Q, dtype=np.float64, copy=True, order="C")
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    _ck(lib().orc_rk3(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), float(dt), int(nsteps)), "rk3")
    return Q


def rk3_jvp(cfg, M, Q, dQ, dt, nsteps=1, dM=None):
    M = _f64(M)
    Q = np.array(Q, dtype=np.float64, copy=True, order="C")
    dQ = np.array(dQ, dtype=np.float64, copy=True, order="C")
    dM = np.zeros_like(M) if dM is None else _f64(dM)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    _ck(lib().orc_rk3_jvp(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(dM), _dp(Q), _dp(dQ),
                          float(dt), int(nsteps)), "rk3_jvp")
    return Q, dQ


def rhs_vjp(cfg, M, Q, g):
    """(Q_bar, M_bar) = (d rhs / d(Q, M))^T g by reverse mode over the oracle's own right-hand
    side (the Rev scalar's tape); M_bar spans the haloed metric array."""
    M, Q, g = _f64(M), _f64(Q), _f64(g)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    Qb, Mb = np.zeros_like(Q), np.zeros_like(M)
    _ck(lib().orc_rhs_vjp(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), _dp(g), _dp(Qb), _dp(Mb)),
        "rhs_vjp")
    return Qb, Mb


def rk3_vjp(cfg, M, Qn, dt, Qbar):
    """Reverse of one RK3 step at Q_n: (dJ/dQ^n, metric adjoint of the step) from
    Qbar = dJ/dQ^{n+1}."""
    M, Qn = _f64(M), _f64(Qn)
    Qb = np.array(Qbar, dtype=np.float64, copy=True, order="C")
    _, nj, ni = Qn.shape
    ip, dp, _ = _params(cfg)
    Mb = np.zeros_like(M)
    _ck(lib().orc_rk3_vjp(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Qn), float(dt), _dp(Qb), _dp(Mb)),
        "rk3_vjp")
    return Qb, Mb


def metrics_vjp(cfg, x, y, Mbar):
    """(x_bar, y_bar) = (d metrics / d(x, y))^T Mbar."""
    x, y, Mbar = _f64(x), _f64(y), _f64(Mbar)
    nj, ni = x.shape
    ip, dp, per = _params(cfg)
    xb, yb = np.zeros_like(x), np.zeros_like(y)
    _ck(lib().orc_metrics_vjp(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(per), _dp(x), _dp(y), _dp(Mbar), _dp(xb),
                              _dp(yb)), "metrics_vjp")
    return xb, yb


def count_vjp_flops(cfg, M, Q):
    """{forward, partials, reverse, records}: operations of one right-hand-side adjoint
    (the forward right-hand side, the partial derivatives its divisions and square roots
    need, and the dense reverse sweep of its tape) and the tape's length."""
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    out = (ctypes.c_longlong * 4)()
    _ck(lib().orc_count_vjp_flops(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), out), "count_vjp_flops")
    return {"forward": out[0], "partials": out[1], "reverse": out[2], "records": out[3]}


def cfl_dt(cfg, M, Q, cfl):
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    return lib().orc_cfl_dt(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), float(cfl))


def count_flops(cfg, M, Q):
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    return int(lib().orc_count_flops(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q)))


def count_char_dir():
    """Operations of one interface's characteristic direction (Section 3.4)."""
    return lib().orc_count_char_dir()


def count_mid_interp(scheme, interp=0):
    """Operations of one midpoint interpolation of a nodal quantity (one metric component)."""
    n = lib().orc_count_mid_interp(int(scheme), int(interp))
    if n < 0:
        raise ValueError("scheme or interpolation option out of range")
    return n


def count_flops_parts(cfg, M, Q):
    """Flops of one right-hand side by part: (lambda_xi, sweep_xi, lambda_eta, sweep_eta, final)."""
    M, Q = _f64(M), _f64(Q)
    _, nj, ni = Q.shape
    ip, dp, _ = _params(cfg)
    out = (ctypes.c_longlong * 5)()
    _ck(lib().orc_count_flops_parts(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(M), _dp(Q), out), "count")
    return tuple(int(v) for v in out)


def fsp_residual(cfg, x, y, q0, wide=False):
    x, y = _f64(x), _f64(y)
    nj, ni = x.shape
    ip, dp, per = _params(cfg)
    q0 = _f64(q0)
    return lib().orc_fsp_residual(ip.ctypes.data_as(_I), _dp(dp), ni, nj, _dp(per), _dp(x), _dp(y),
                                  _dp(q0), int(bool(wide)))


def weno(r, u, ppm=1, linw=0, eps=1e-40):
    """WENO interpolation to x_{j+1/2} from u_{j-2..j+2} (5 values) or u_{j-3..j+3} (7)."""
    u = _f64(u)
    if u.size == 5:
        u = np.concatenate(([0.0], u, [0.0]))
    return lib().orc_weno(int(r), int(ppm), int(linw), float(eps), _dp(u))


def ppm(order, w, C):
    return lib().orc_ppm(int(order), float(w), float(C))


def smoothness(u5):
    u5 = _f64(u5)
    out = np.empty(3)
    lib().orc_smoothness(_dp(u5), _dp(out))
    return out


def eig(gamma, q, nx, ny):
    q = _f64(q)
    L, R = np.empty((4, 4)), np.empty((4, 4))
    lib().orc_eig(float(gamma), _dp(q), float(nx), float(ny), _dp(L), _dp(R))
    return L, R


def scheme_table(scheme, alpha=1.0):
    """r, h+ midpoint coefficients (m = 0, -1), h+ node coefficients of f_{j+k} (k = -3..3),
    central-operator node coefficients a_k (k = 1..4) and midpoint coefficients (1/2, 3/2); for
    the four-midpoint scheme also the h+ coefficients of f_{j+1/2+m}, m = -2, +1 (hmidx) and the
    central operator's 5/2 coefficient (cmid3); alpha: the free parameter of the one-midpoint
    forms."""
    out = np.empty(19)
    lib().orc_scheme_table(int(scheme), float(alpha), _dp(out))
    return {"r": int(out[0]), "hmid": out[1:3], "hnode": out[3:10], "cnode": out[10:14], "cmid": out[14:16],
            "hmidx": out[16:18], "cmid3": float(out[18])}


def smoothness4(u7):
    """The four r = 4 indicators of u_{j-3..j+3}."""
    u7 = _f64(u7)
    out = np.empty(4)
    lib().orc_smoothness4(_dp(u7), _dp(out))
    return out


def advect1d_dt(scheme, N, dt_exp, tfinal=2.0):
    out = np.empty(3)
    _ck(lib().orc_advect1d_dt(int(scheme), int(N), float(tfinal), float(dt_exp), _dp(out)), "advect1d_dt")
    return out[0], out[1], int(out[2])


def advect1d_opts(scheme, N, tfinal=2.0, dt_exp=1.25, weights=0):
    """Scalar advection (Table 3 setup) with the weight option (1: WENO-Z)."""
    out = np.empty(3)
    _ck(lib().orc_advect1d_opts(int(scheme), int(N), float(tfinal), float(dt_exp), int(weights), _dp(out)),
        "advect1d_opts")
    return out[0], out[1], int(out[2])


def weno_z(r, eps, u7):
    """WENO-Z interpolation to x_{j+1/2} of u7[m + 3] = u_{j+m}."""
    return float(lib().orc_weno_z(int(r), float(eps), _dp(_f64(u7))))


def split_flux(mode, q, mx, my, gamma=1.4):
    """(F+, F-, E^) of the midpoint splitting `mode` (1 Steger-Warming, 2 Van Leer)."""
    q = _f64(np.asarray(q).reshape(4))
    fp, fm, e = np.empty(4), np.empty(4), np.empty(4)
    _ck(lib().orc_split_flux(int(mode), _dp(q), float(mx), float(my), float(gamma), _dp(fp), _dp(fm), _dp(e)),
        "split_flux")
    return fp, fm, e


def advect1d(scheme, N, tfinal=2.0):
    out = np.empty(3)
    _ck(lib().orc_advect1d(int(scheme), int(N), float(tfinal), _dp(out)), "advect1d")
    return out[0], out[1], int(out[2])


def riemann_exact(gamma, left, right, x0, t, x):
    x = _f64(x)
    L, R = _f64(left), _f64(right)
    out = np.empty((x.size, 3))
    lib().orc_riemann_exact(float(gamma), _dp(L), _dp(R), float(x0), float(t), x.size, _dp(x), _dp(out))
    return out


def long_double_digits():
    return int(lib().orc_long_double_digits())


# ---------------------------------------------------------------------------------------
# Multi-block grids.  `blocks` is a list of dicts with keys x, y (nj, ni), bc (4 codes, 5 =
# linked face), links (4 entries, each None or (nbr, face, reversed)), offsets (4 entries
# (dx, dy) or None, added to ghost coordinates across the link), period (as for one block).
# ---------------------------------------------------------------------------------------
def _mb_tables(blocks):
    nb = len(blocks)
    dims = np.array([[b["x"].shape[1], b["x"].shape[0]] for b in blocks], dtype=np.int32).reshape(-1)
    bcs = np.array([list(b["bc"]) for b in blocks], dtype=np.int32).reshape(-1)
    lk = np.full((nb, 4, 3), -1, dtype=np.int32)
    off = np.zeros((nb, 4, 2))
    per = np.zeros((nb, 4))
    for k, b in enumerate(blocks):
        for f in range(4):
            l = (b.get("links") or [None] * 4)[f]
            if l is not None:
                lk[k, f] = l
            o = (b.get("offsets") or [None] * 4)[f]
            if o is not None:
                off[k, f] = o
        per[k] = np.asarray(b.get("period", ((0.0, 0.0), (0.0, 0.0))), dtype=np.float64).reshape(4)
    return nb, dims, bcs, lk.reshape(-1), off.reshape(-1), per.reshape(-1)


def mb_metrics(cfg, blocks):
    nb, dims, bcs, lk, off, per = _mb_tables(blocks)
    ip, dp, _ = _params(cfg)
    x = np.concatenate([_f64(b["x"]).reshape(-1) for b in blocks])
    y = np.concatenate([_f64(b["y"]).reshape(-1) for b in blocks])
    sizes = [5 * (b["x"].shape[0] + 2 * G) * (b["x"].shape[1] + 2 * G) for b in blocks]
    M = np.empty(sum(sizes))
    _ck(lib().orc_mb_metrics(ip.ctypes.data_as(_I), _dp(dp), nb, dims.ctypes.data_as(_I), bcs.ctypes.data_as(_I),
                             lk.ctypes.data_as(_I), _dp(off), _dp(per), _dp(x), _dp(y), _dp(M)), "mb_metrics")
    out, o = [], 0
    for b, n in zip(blocks, sizes):
        out.append(M[o:o + n].reshape(5, b["x"].shape[0] + 2 * G, b["x"].shape[1] + 2 * G))
        o += n
    return out


def _mb_state(blocks, Qs):
    return np.concatenate([_f64(q).reshape(-1) for q in Qs])


def mb_rhs(cfg, blocks, Ms, Qs):
    nb, dims, bcs, lk, _, _ = _mb_tables(blocks)
    ip, dp, _ = _params(cfg)
    M = np.concatenate([_f64(m).reshape(-1) for m in Ms])
    Q = _mb_state(blocks, Qs)
    R = np.empty_like(Q)
    _ck(lib().orc_mb_rhs(ip.ctypes.data_as(_I), _dp(dp), nb, dims.ctypes.data_as(_I), bcs.ctypes.data_as(_I),
                         lk.ctypes.data_as(_I), _dp(M), _dp(Q), _dp(R)), "mb_rhs")
    out, o = [], 0
    for q in Qs:
        out.append(R[o:o + q.size].reshape(q.shape))
        o += q.size
    return out


def mb_rk3(cfg, blocks, Ms, Qs, dt, nsteps=1):
    nb, dims, bcs, lk, _, _ = _mb_tables(blocks)
    ip, dp, _ = _params(cfg)
    M = np.concatenate([_f64(m).reshape(-1) for m in Ms])
    Q = _mb_state(blocks, Qs).copy()
    _ck(lib().orc_mb_rk3(ip.ctypes.data_as(_I), _dp(dp), nb, dims.ctypes.data_as(_I), bcs.ctypes.data_as(_I),
                         lk.ctypes.data_as(_I), _dp(M), _dp(Q), float(dt), int(nsteps)), "mb_rk3")
    out, o = [], 0
    for q in Qs:
        out.append(Q[o:o + q.size].reshape(q.shape))
        o += q.size
    return out


# ---- three dimensions ------------------------------------------------------------------------
# cfg keys as above, with ``bc`` six face codes (i-min, i-max, j-min, j-max, k-min, k-max: 0
# periodic, 1 transmissive) and ``period`` three vectors (added per wrap in i, j, k).  Arrays:
# coordinates (nk, nj, ni); state (5, nk, nj, ni); metrics (10, nk+8, nj+8, ni+8): the planes
# xi_x^, xi_y^, xi_z^, eta_x^, eta_y^, eta_z^, zeta_x^, zeta_y^, zeta_z^, J^-1.
def _params3(cfg):
    ip = np.array([cfg.get("scheme", 2), cfg.get("interp", 0), cfg.get("ppm", 1), cfg.get("linear_weights", 0)]
                  + list(cfg.get("bc", (0, 0, 0, 0, 0, 0))), dtype=np.int32)
    per = np.asarray(cfg.get("period", ((0.0,) * 3,) * 3), dtype=np.float64).reshape(9)
    dp = np.concatenate([[cfg.get("gamma", 1.4), cfg.get("lf_alpha", 1.1), cfg.get("eps", 1e-40)], per])
    return ip, dp.astype(np.float64)


def metrics3(cfg, x, y, z):
    ip, dp = _params3(cfg)
    nk, nj, ni = x.shape
    M = np.zeros((10, nk + 2 * G, nj + 2 * G, ni + 2 * G))
    _ck(lib().orc3_metrics(ip.ctypes.data_as(_I), _dp(dp), ni, nj, nk, _dp(_f64(x)), _dp(_f64(y)), _dp(_f64(z)),
                           _dp(M)), "metrics3")
    return M


def rhs3(cfg, M, Q):
    ip, dp = _params3(cfg)
    _, nk, nj, ni = Q.shape
    R = np.zeros_like(Q, dtype=np.float64)
    _ck(lib().orc3_rhs(ip.ctypes.data_as(_I), _dp(dp), ni, nj, nk, _dp(_f64(M)), _dp(_f64(Q)), _dp(R)), "rhs3")
    return R


def rk3_3(cfg, M, Q, dt, nsteps=1):
    ip, dp = _params3(cfg)
    _, nk, nj, ni = Q.shape
    out = np.array(Q, dtype=np.float64, copy=True)
    _ck(lib().orc3_rk3(ip.ctypes.data_as(_I), _dp(dp), ni, nj, nk, _dp(_f64(M)), _dp(out), float(dt), int(nsteps)),
        "rk3_3")
    return out


def lambda3(cfg, M, Q, d):
    """A^ of every line of direction d (0 xi, 1 eta, 2 zeta), shape (n2, n1): the other two
    indices in the order (i, j, k) with the first fastest."""
    ip, dp = _params3(cfg)
    _, nk, nj, ni = Q.shape
    n = (ni, nj, nk)
    others = [n[a] for a in range(3) if a != d]
    out = np.zeros((others[1], others[0]))
    _ck(lib().orc3_lambda(ip.ctypes.data_as(_I), _dp(dp), ni, nj, nk, int(d), _dp(_f64(M)), _dp(_f64(Q)), _dp(out)),
        "lambda3")
    return out


def count_flops3(cfg, M, Q):
    """Operations of one right-hand side and of its xi, eta and zeta sweeps."""
    ip, dp = _params3(cfg)
    _, nk, nj, ni = Q.shape
    out = (ctypes.c_longlong * 4)()
    _ck(lib().orc3_count_flops(ip.ctypes.data_as(_I), _dp(dp), ni, nj, nk, _dp(_f64(M)), _dp(_f64(Q)), out),
        "count_flops3")
    return dict(rhs=out[0], xi=out[1], eta=out[2], zeta=out[3])


def eig3(gamma, q, n):
    L, R = np.zeros((5, 5)), np.zeros((5, 5))
    lib().orc3_eig(float(gamma), _dp(_f64(q)), _dp(_f64(n)), _dp(L), _dp(R))
    return L, R


def fsp_residual3(cfg, x, y, z, q0, wide=False):
    ip, dp = _params3(cfg)
    nk, nj, ni = x.shape
    r = lib().orc3_fsp_residual(ip.ctypes.data_as(_I), _dp(dp), ni, nj, nk, _dp(_f64(x)), _dp(_f64(y)),
                                _dp(_f64(z)), _dp(_f64(q0)), int(bool(wide)))
    if r < 0:
        raise ValueError("oracle fsp_residual3: invalid arguments")
    return r
