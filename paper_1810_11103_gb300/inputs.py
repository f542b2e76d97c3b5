"""Seeded synthetic inputs: grids and initial states shaped like the paper's test cases.

This module holds no arithmetic of the method (no metrics, fluxes, interpolation or
time stepping).  It only draws random numbers and writes coordinates and initial states,
so both the CPU oracle and the CUDA path can be fed the same inputs.

Random numbers: splitmix64 of ``seed ^ (block << 32) ^ (4 * node + draw)`` mapped to a
double in [0, 1) by ``(z >> 11) * 2**-53``.  ``node`` is the flat index j * ni + i,
``draw`` is 0 (x offset), 1 (y offset) or 2 (the coin, bit 0 of the draw).

Randomised grids follow Section 6.1 (1): every node moves along one coordinate only,
chosen by a fair coin, by h * 2A (r - 1/2).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied element-wise to uint64 keys (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def _keys(seed: int, block: int, n: int, draw: int) -> np.ndarray:
    node = np.arange(n, dtype=np.uint64)
    base = np.uint64(seed) ^ (np.uint64(block) << np.uint64(32))
    return base ^ (np.uint64(4) * node + np.uint64(draw))


def uniform(seed: int, block: int, n: int, draw: int) -> np.ndarray:
    """n uniform doubles in [0, 1) for nodes 0..n-1."""
    z = splitmix64(_keys(seed, block, n, draw))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def coin(seed: int, block: int, n: int) -> np.ndarray:
    """n fair bits (0/1) for nodes 0..n-1."""
    z = splitmix64(_keys(seed, block, n, 2))
    return (z & np.uint64(1)).astype(np.float64)


def randomize(x: np.ndarray, y: np.ndarray, hx: float, hy: float, amp: np.ndarray, seed: int,
              block: int = 0):
    """Perturb a grid as in Section 6.1 (1): one coordinate per node, chosen by a coin."""
    nj, ni = x.shape
    n = ni * nj
    r1 = uniform(seed, block, n, 0).reshape(nj, ni)
    r2 = uniform(seed, block, n, 1).reshape(nj, ni)
    b = coin(seed, block, n).reshape(nj, ni)
    xr = x + hx * 2.0 * amp * (r1 - 0.5) * b
    yr = y + hy * 2.0 * amp * (r2 - 0.5) * (1.0 - b)
    return xr, yr


def periodic_square(n: int, length: float, amp: float, seed: int, origin=(0.0, 0.0), nj: int | None = None):
    """n x nj unique nodes of a periodic box [origin, origin + length)^2, every node
    randomised with amplitude ``amp`` (fraction of the spacing).  Returns x, y, period."""
    nj = n if nj is None else nj
    hx, hy = length / n, length / nj
    i = np.arange(n, dtype=np.float64)
    j = np.arange(nj, dtype=np.float64)
    x = np.broadcast_to(origin[0] + hx * i[None, :], (nj, n)).copy()
    y = np.broadcast_to(origin[1] + hy * j[:, None], (nj, n)).copy()
    if amp > 0:
        x, y = randomize(x, y, hx, hy, np.full((nj, n), amp), seed)
    period = ((length, 0.0), (0.0, length))
    return x, y, period


def paper_random_grid(imax: int, jmax: int, length: float, amp: float, seed: int, margin: int = 4):
    """The grid of Section 6.1 (1): [-L/2, L/2]^2 with imax x jmax nodes, nodes of the
    interior window (1-based i = 5..imax-4 and j = 5..jmax-4 for margin 4) randomised."""
    h = length / (imax - 1)
    i = np.arange(imax, dtype=np.float64)
    j = np.arange(jmax, dtype=np.float64)
    x = np.broadcast_to(-length / 2 + h * i[None, :], (jmax, imax)).copy()
    y = np.broadcast_to(-length / 2 + h * j[:, None], (jmax, imax)).copy()
    A = np.zeros((jmax, imax))
    A[margin:jmax - margin, margin:imax - margin] = amp
    x, y = randomize(x, y, h, h, A, seed)
    return x, y


def curved_periodic(n: int, length: float, warp: float = 0.1, origin=(0.0, 0.0)):
    """A smooth curved periodic grid: x = xi + warp L/(2 pi) sin(2 pi xi/L) sin(2 pi eta/L),
    y likewise (both perturbations periodic).  Returns x, y, period."""
    h = length / n
    s = origin[0] + h * np.arange(n, dtype=np.float64)
    t = origin[1] + h * np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(s, t)
    k = 2.0 * math.pi / length
    a = warp / k
    x = X + a * np.sin(k * (X - origin[0])) * np.sin(k * (Y - origin[1]))
    y = Y + a * np.sin(k * (X - origin[0])) * np.sin(k * (Y - origin[1]))
    return x, y, ((length, 0.0), (0.0, length))


# ----------------------------------------------------------------------------------------
# Initial states (conservative variables Q = (rho, rho u, rho v, E), E = p/(g-1) + rho|u|^2/2)
# ----------------------------------------------------------------------------------------
def conservative(rho, u, v, p, gamma: float = GAMMA) -> np.ndarray:
    rho, u, v, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, u, v, p)))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def uniform_state(shape, rho=1.0, u=1.0, v=1.0, p=1.0, gamma: float = GAMMA) -> np.ndarray:
    nj, ni = shape
    return conservative(np.full((nj, ni), rho), np.full((nj, ni), u), np.full((nj, ni), v),
                        np.full((nj, ni), p), gamma)


def isentropic_vortex(x, y, center, strength=5.0, free=(1.0, 1.0, 1.0, 1.0), period=None,
                      alpha=0.5, rc=1.0, gamma: float = GAMMA) -> np.ndarray:
    """Isentropic vortex of Section 6.3 (1) on a free stream (rho, u, v, p); the paper's
    epsilon is strength / (2 pi).  With ``period`` = (Lx, Ly) the nearest periodic image
    of the centre is used."""
    rho0, u0, v0, p0 = free
    dx = x - center[0]
    dy = y - center[1]
    if period is not None:
        dx = dx - period[0] * np.round(dx / period[0])
        dy = dy - period[1] * np.round(dy / period[1])
    r2 = (dx * dx + dy * dy) / (rc * rc)
    eps = strength / (2.0 * math.pi)
    e = np.exp(alpha * (1.0 - r2))
    # (du, dv) = eps r e^{alpha(1 - r^2)} (sin theta, -cos theta) = eps e (dy, -dx)
    du = eps * e * dy / rc
    dv = -eps * e * dx / rc
    T0 = p0 / rho0
    dT = -(gamma - 1.0) * eps * eps / (4.0 * alpha * gamma) * e * e
    T = T0 + dT
    S0 = p0 / rho0 ** gamma
    rho = (T / S0) ** (1.0 / (gamma - 1.0))     # isentropic: T = p/rho = S0 rho^(g-1)
    p = rho * T
    return conservative(rho, u0 + du, v0 + dv, p, gamma)


def sod_1d(n: int = 200, gamma: float = GAMMA):
    """Sod tube on [0, 1] with n cell-centred nodes, interface at 0.5: left (1, 0, 1),
    right (0.125, 0, 0.1).  Returns x (1, n), y (1, n), Q (4, 1, n), period."""
    xs = (np.arange(n, dtype=np.float64) + 0.5) / n
    left = xs < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    Q = conservative(rho[None, :], np.zeros((1, n)), np.zeros((1, n)), p[None, :], gamma)
    x = xs[None, :].copy()
    y = np.zeros((1, n))
    period = ((0.0, 0.0), (0.0, 1.0 / n))
    return x, y, Q, period


def riemann_quadrants(x, y, gamma: float = GAMMA) -> np.ndarray:
    """Four-quadrant state on [0, 1]^2 split at 0.5, quadrants in the paper's order
    (upper right, upper left, lower left, lower right)."""
    states = {
        "ur": (1.5, 0.0, 0.0, 1.5),
        "ul": (0.5323, 1.206, 0.0, 0.3),
        "ll": (0.138, 1.206, 1.206, 0.029),
        "lr": (0.5323, 0.0, 1.206, 0.3),
    }
    right = x >= 0.5
    up = y >= 0.5
    out = np.zeros((4,) + x.shape)
    for key, mask in (("ur", right & up), ("ul", ~right & up), ("ll", ~right & ~up), ("lr", right & ~up)):
        q = conservative(*(np.full(x.shape, c) for c in states[key]), gamma=gamma)
        out[:, mask] = q[:, mask]
    return out


def riemann_grid(n: int, amp: float, seed: int, lo: float = 0.25, hi: float = 0.75):
    """[0, 1]^2 with n x n nodes, nodes inside the central square [lo, hi]^2 randomised."""
    h = 1.0 / (n - 1)
    s = h * np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(s, s)
    A = np.where((X > lo) & (X < hi) & (Y > lo) & (Y < hi), amp, 0.0)
    return randomize(X, Y, h, h, A, seed)


def random_state(shape, seed: int, rho=(0.8, 1.2), vel=(-0.3, 0.3), p=(0.8, 1.2),
                 gamma: float = GAMMA, block: int = 7) -> np.ndarray:
    """A smooth-free random state (every node independent) for algebraic tests."""
    nj, ni = shape
    n = ni * nj
    r = [uniform(seed, block + k, n, 0).reshape(nj, ni) for k in range(4)]
    return conservative(rho[0] + (rho[1] - rho[0]) * r[0], vel[0] + (vel[1] - vel[0]) * r[1],
                        vel[0] + (vel[1] - vel[0]) * r[2], p[0] + (p[1] - p[0]) * r[3], gamma)


# ----------------------------------------------------------------------------------------
# Multi-block grids
# ----------------------------------------------------------------------------------------
LINK = 5


def split_blocks(x, y, q, isplit, jsplit, bc_outer, period=None):
    """Cut one (nj, ni) grid into blocks at the i indices `isplit` and j indices `jsplit`
    (interior cut points).  Faces between blocks are linked; the outer faces keep
    bc_outer (i-min, i-max, j-min, j-max), periodic outer faces becoming links that wrap
    (with the period vector as the coordinate offset).  Returns (blocks, states)."""
    nj, ni = x.shape
    ic = [0] + list(isplit) + [ni]
    jc = [0] + list(jsplit) + [nj]
    na, nbk = len(ic) - 1, len(jc) - 1
    per = period if period is not None else ((0.0, 0.0), (0.0, 0.0))
    blocks, states = [], []
    idx = lambda a, b: b * na + a
    for b in range(nbk):
        for a in range(na):
            sl = (slice(jc[b], jc[b + 1]), slice(ic[a], ic[a + 1]))
            bc, links, offs = [0] * 4, [None] * 4, [None] * 4
            # i-min / i-max
            for f, (da, outer) in enumerate(((-1, a == 0), (1, a == na - 1))):
                if not outer:
                    bc[f], links[f] = LINK, (idx(a + da, b), 1 - f, 0)
                elif bc_outer[f] == 0:
                    bc[f], links[f] = LINK, (idx((a + da) % na, b), 1 - f, 0)
                    offs[f] = (da * per[0][0], da * per[0][1])
                else:
                    bc[f] = bc_outer[f]
            for f, (db, outer) in ((2, (-1, b == 0)), (3, (1, b == nbk - 1))):
                if not outer:
                    bc[f], links[f] = LINK, (idx(a, b + db), 5 - f, 0)
                elif bc_outer[f] == 0:
                    bc[f], links[f] = LINK, (idx(a, (b + db) % nbk), 5 - f, 0)
                    offs[f] = (db * per[1][0], db * per[1][1])
                else:
                    bc[f] = bc_outer[f]
            blocks.append({"x": x[sl].copy(), "y": y[sl].copy(), "bc": bc, "links": links, "offsets": offs,
                           "period": ((0.0, 0.0), (0.0, 0.0))})
            states.append(None if q is None else q[(slice(None),) + sl].copy())
    return blocks, states


def cylinder_blocks(seed=1812, cols=8, rows=8, imin=64, imax=512, jmin=64, jmax=384, step=32,
                    r_in=0.5, r_out=6.0, stretch=1.002, frac_random=0.3, amp=0.2, margin=4,
                    mach=4.0, gamma: float = GAMMA):
    """Body-fitted polar blocks around a cylinder of diameter one: `cols` angular columns of
    I_a nodes and `rows` radial rows of J_b nodes (sizes drawn from the seed, multiples of
    `step`), so blocks are uneven but shared faces match node for node.  Angle runs
    clockwise so the grid is right-handed; radius is geometrically stretched from r_in to
    r_out.  A seeded `frac_random` of the blocks is randomised with amplitude `amp` away
    from a `margin`-node frame.  Faces: slip wall at r_in, far field at r_out (free stream
    Mach `mach` along +x), links elsewhere (the angular direction wraps).
    Returns (blocks, states, free_state)."""
    rng_i = uniform(seed, 900, cols, 0)
    rng_j = uniform(seed, 901, rows, 0)
    I = [imin + step * int(r * ((imax - imin) // step + 1)) for r in rng_i]
    J = [jmin + step * int(r * ((jmax - jmin) // step + 1)) for r in rng_j]
    nth, nr = sum(I), sum(J)
    th = 2.0 * math.pi * np.arange(nth) / nth
    m = np.arange(nr, dtype=np.float64)
    rr = r_in + (r_out - r_in) * (stretch ** m - 1.0) / (stretch ** (nr - 1) - 1.0)
    TH, RR = np.meshgrid(th, rr)
    x = RR * np.cos(TH)
    y = -RR * np.sin(TH)
    free = conservative(1.0, mach, 0.0, 1.0 / gamma, gamma)
    q = np.broadcast_to(free[:, None, None], (4, nr, nth)).copy()
    blocks, states = split_blocks(x, y, q, np.cumsum(I)[:-1], np.cumsum(J)[:-1],
                                  (0, 0, BC_WALL, BC_FAR))
    pick = uniform(seed, 902, len(blocks), 0) < frac_random
    for k, b in enumerate(blocks):
        b["bc_state"] = [list(free)] * 4
        if pick[k]:
            nj, ni = b["x"].shape
            A = np.zeros((nj, ni))
            A[margin:nj - margin, margin:ni - margin] = amp
            b["x"], b["y"] = randomize_local(b["x"], b["y"], A, seed, block=1000 + k)
    return blocks, states, free


BC_WALL, BC_FAR = 3, 4


def randomize_local(x, y, amp, seed, block=0):
    """Section 6.1 (1) randomisation on a curved block: each node moves by 2A (r - 1/2)
    times the local spacing along one grid direction (a coin picks which)."""
    nj, ni = x.shape
    n = ni * nj
    r1 = uniform(seed, block, n, 0).reshape(nj, ni)
    r2 = uniform(seed, block, n, 1).reshape(nj, ni)
    b = coin(seed, block, n).reshape(nj, ni)
    dxi = (np.gradient(x, axis=1), np.gradient(y, axis=1))
    deta = (np.gradient(x, axis=0), np.gradient(y, axis=0))
    s1 = 2.0 * amp * (r1 - 0.5) * b
    s2 = 2.0 * amp * (r2 - 0.5) * (1.0 - b)
    return x + s1 * dxi[0] + s2 * deta[0], y + s1 * dxi[1] + s2 * deta[1]


# ----------------------------------------------------------------------------------------
# Shock-vortex interaction (Section 6.3 (4)) on a smooth stretched grid
# ----------------------------------------------------------------------------------------
def _sinh_map(n: int, lo: float, hi: float, beta: float):
    """n nodes on [lo, hi] clustered around 0 by x = c sinh(beta (s - s0)), s uniform in
    [0, 1]; s0 and c are fixed by x(0) = lo, x(1) = hi (lo < 0 < hi).  The ratio of
    neighbouring spacings is at most exp(beta / (n - 1))."""
    a, b = 0.0, 1.0
    for _ in range(200):                      # bisection on sinh(beta s0) / sinh(beta (1 - s0)) = -lo / hi
        s0 = 0.5 * (a + b)
        if math.sinh(beta * s0) * hi < -lo * math.sinh(beta * (1.0 - s0)):
            a = s0
        else:
            b = s0
    c = hi / math.sinh(beta * (1.0 - s0))
    s = np.arange(n, dtype=np.float64) / (n - 1)
    x = c * np.sinh(beta * (s - s0))
    x[0], x[-1] = lo, hi
    return s, x, c * beta * np.cosh(beta * (s - s0)) / (n - 1)


def shock_vortex_grid(n: int = 512, nj: int | None = None, lo=(-20.0, -15.0), hi=(10.0, 15.0),
                      beta: float = 3.0, warp: float = 0.1, waves: int = 4):
    """The domain of Section 6.3 (4), [-20, 10] x [-15, 15], with x(xi) clustered at the
    shock (x = 0) and y(eta) at y = 0 by a sinh stretching, plus a smooth warp of
    ``warp`` times the local spacing, sin(2 pi waves s) sin(2 pi waves t) in both
    coordinates, which vanishes on the four boundaries.  Returns x, y of shape (nj, n)."""
    nj = n if nj is None else nj
    s, xs, hx = _sinh_map(n, lo[0], hi[0], beta)
    t, ys, hy = _sinh_map(nj, lo[1], hi[1], beta)
    w = np.sin(2.0 * math.pi * waves * s)[None, :] * np.sin(2.0 * math.pi * waves * t)[:, None]
    x = xs[None, :] + warp * hx[None, :] * w
    y = ys[:, None] + warp * hy[:, None] * w
    return x, y


def shock_vortex_state(x, y, mach: float = 1.1, strength: float = 0.4, center=(4.0, 0.0),
                       gamma: float = GAMMA) -> np.ndarray:
    """Stationary normal shock at x = 0 with an isentropic vortex ahead of it (Section 6.3
    (4)).  Upstream (x > 0): (rho, u, v, p) = (1, -1, 0, 1/(gamma M^2)); downstream from the
    Rankine-Hugoniot relations.  Vortex: u_theta = G r e^{(1 - r^2)/2},
    T = 1 - (gamma - 1)/2 M^2 G^2 e^{1 - r^2}, rho = T^{1/(gamma-1)}, p = rho T/(gamma M^2)
    (the M^2 factor makes dp/dr = rho u_theta^2 / r hold)."""
    m2 = mach * mach
    p1 = 1.0 / (gamma * m2)
    rho2 = (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    u2 = -1.0 / rho2
    dx, dy = x - center[0], y - center[1]
    e = np.exp(1.0 - dx * dx - dy * dy)
    T = 1.0 - 0.5 * (gamma - 1.0) * m2 * strength * strength * e
    rho_v = T ** (1.0 / (gamma - 1.0))
    g = strength * np.sqrt(e)                  # u_theta / r
    up = x > 0.0
    rho = np.where(up, rho_v, rho2)
    u = np.where(up, -1.0 - g * dy, u2)
    v = np.where(up, g * dx, 0.0)
    p = np.where(up, rho_v * T * p1, p2)
    return conservative(rho, u, v, p, gamma)


def shock_vortex_bc(mach: float = 1.1, gamma: float = GAMMA):
    """Boundary kinds and states of the shock-vortex case: transmissive outflow at x = -20
    (face 0), the upstream state imposed at x = 10 (face 1), transmissive at y = +-15."""
    up = conservative(1.0, -1.0, 0.0, 1.0 / (gamma * mach * mach), gamma)
    return (1, 2, 1, 1), np.tile(up, (4, 1))


def smooth_field(shape, seed: int, modes: int = 3, block: int = 11) -> np.ndarray:
    """A smooth random field on an (nj, ni) index grid: a sum of modes x modes products of
    sines with seeded amplitudes and phases, peak value about 1."""
    nj, ni = shape
    r = uniform(seed, block, 4 * modes * modes, 0)
    s = np.arange(ni, dtype=np.float64) / max(ni - 1, 1)
    t = np.arange(nj, dtype=np.float64) / max(nj - 1, 1)
    out = np.zeros((nj, ni))
    for a in range(modes):
        for b in range(modes):
            k = 4 * (a * modes + b)
            amp, ph1, ph2 = 2.0 * r[k] - 1.0, 2.0 * math.pi * r[k + 1], 2.0 * math.pi * r[k + 2]
            out += amp * np.sin(math.pi * (a + 1) * s + ph1)[None, :] * np.sin(math.pi * (b + 1) * t + ph2)[:, None]
    return out / max(np.abs(out).max(), 1e-300)


# ----------------------------------------------------------------------------------------
# The paper's own test problems (Sections 6.1-6.3), at the paper's sizes
# ----------------------------------------------------------------------------------------
def _line_1d(n: int, lo: float, hi: float):
    """n uniform nodes on [lo, hi] (both ends included) as a single periodic row."""
    xs = lo + (hi - lo) * np.arange(n, dtype=np.float64) / (n - 1)
    return xs[None, :].copy(), np.zeros((1, n)), ((0.0, 0.0), (0.0, (hi - lo) / (n - 1)))


def paper_sod(n: int = 100, gamma: float = GAMMA):
    """Section 6.2 (1): [-5, 5] with n uniform nodes; (rho, u, p) = (0.125, 0, 0.1) for
    x < 0 and (1, 0, 1) for x >= 0 (the low-pressure side on the left); the paper runs to
    t = 2 with dt = 0.01.  Returns x (1, n), y (1, n), Q (4, 1, n), period."""
    x, y, per = _line_1d(n, -5.0, 5.0)
    left = x < 0.0
    Q = conservative(np.where(left, 0.125, 1.0), np.zeros_like(x), np.zeros_like(x), np.where(left, 0.1, 1.0),
                     gamma)
    return x, y, Q, per


def shu_osher(n: int = 400, gamma: float = GAMMA):
    """Section 6.2 (2): [-5, 5] with n uniform nodes; (rho, u, p) = (3.857143, 2.629369,
    10.3333) for x < -4 and (1 + 0.2 sin 5x, 0, 1) for x >= -4; the paper runs to t = 1.8
    with dt = 0.001.  Returns x (1, n), y (1, n), Q (4, 1, n), period."""
    x, y, per = _line_1d(n, -5.0, 5.0)
    left = x < -4.0
    Q = conservative(np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x)), np.where(left, 2.629369, 0.0),
                     np.zeros_like(x), np.where(left, 10.3333, 1.0), gamma)
    return x, y, Q, per


def paper_vortex_grid(imax: int = 81, length: float = 16.0, amp: float = 0.45, seed: int = 1814,
                      randomized: bool = True):
    """Section 6.1 (1) with the periodic boundaries of Section 6.3 (1): the imax x imax grid
    lines of [-L/2, L/2]^2, whose last line is the periodic image of the first, so imax - 1
    unique nodes per direction (h = L/(imax - 1)); nodes of the window 1-based i, j =
    5..imax-4 moved by the formula of Section 6.1 (1) with A = amp.  Returns x, y, period."""
    n = imax - 1
    h = length / n
    s = -length / 2 + h * np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(s, s)
    if randomized:
        A = np.zeros((n, n))
        A[4:imax - 4, 4:imax - 4] = amp
        X, Y = randomize(X, Y, h, h, A, seed)
    return X, Y, ((length, 0.0), (0.0, length))


def paper_vortex_state(x, y, period, gamma: float = GAMMA) -> np.ndarray:
    """Section 6.3 (1): free stream of density 1 and sound speed 1 (p = 1/gamma) at Mach 1
    along +x, with the isentropic vortex at the origin (r_c = 1, alpha = 0.204,
    epsilon = 0.3).  Over t = 16 (one period of the L = 16 box) it returns to its start."""
    L = period[0][0]
    return isentropic_vortex(x, y, (0.0, 0.0), strength=0.3 * 2.0 * math.pi, free=(1.0, 1.0, 0.0, 1.0 / gamma),
                             period=(L, L), alpha=0.204, rc=1.0, gamma=gamma)


def paper_cylinder(imax: int = 121, jmax: int = 41, randomized: bool = True, seed: int = 1815, amp: float = 0.2,
                   r_body: float = 0.5, outer=(1.6, 3.2), mach: float = 4.0, gamma: float = GAMMA):
    """Section 6.1 (2): the upstream half of a cylinder of diameter one in a Mach 4 stream
    along +x, imax streamwise x jmax wall-normal nodes.  The smooth grid is the ordinary
    transfinite (linear) interpolation between the body, r = 0.5 for theta from 270 down to
    90 degrees, and an outer ellipse (semi-axes outer[0] along x, outer[1] along y) that holds
    the bow shock; the randomised grid moves the nodes of the window (6, imax - 5) x
    (7, jmax - 6) (1-based) by amp times the local spacing along one grid direction.
    Faces: i-min and i-max transmissive (supersonic outflow), j-min slip wall, j-max far
    field (the free stream enters).  Free stream: rho = 1, p = 1/gamma, u = mach.
    Returns x, y, bc, bc_state."""
    # theta from 270 down to 90 degrees: with the wall-normal index outward the grid is right-handed
    th = 1.5 * math.pi - math.pi * np.arange(imax, dtype=np.float64) / (imax - 1)
    s = np.arange(jmax, dtype=np.float64) / (jmax - 1)
    xb, yb = r_body * np.cos(th), r_body * np.sin(th)
    xo, yo = outer[0] * np.cos(th), outer[1] * np.sin(th)
    x = (1.0 - s)[:, None] * xb[None, :] + s[:, None] * xo[None, :]
    y = (1.0 - s)[:, None] * yb[None, :] + s[:, None] * yo[None, :]
    if randomized:
        A = np.zeros((jmax, imax))
        A[6:jmax - 6, 5:imax - 5] = amp
        x, y = randomize_local(x, y, A, seed)
    free = conservative(1.0, mach, 0.0, 1.0 / gamma, gamma)
    return x, y, (1, 1, BC_WALL, BC_FAR), np.tile(free, (4, 1))


def _box_grid(n: int, lo, hi, amp: float, margin: int, seed: int, randomized: bool):
    """n x n grid lines of the box [lo, hi]; with `randomized`, the nodes more than `margin`
    layers inside the boundary moved by the formula of Section 6.1 (1) (h = the spacing)."""
    hx, hy = (hi[0] - lo[0]) / (n - 1), (hi[1] - lo[1]) / (n - 1)
    X, Y = np.meshgrid(lo[0] + hx * np.arange(n, dtype=np.float64), lo[1] + hy * np.arange(n, dtype=np.float64))
    if randomized:
        A = np.zeros((n, n))
        A[margin:n - margin, margin:n - margin] = amp
        X, Y = randomize(X, Y, hx, hy, A, seed)
    return X, Y


def paper_riemann_grid(n: int = 401, randomized: bool = True, seed: int = 1816):
    """Section 6.1 (3): [0, 1]^2 with n x n grid lines (the paper's 400 x 400 cells), four
    uniform layers at the boundaries, A = 0.2 inside."""
    return _box_grid(n, (0.0, 0.0), (1.0, 1.0), 0.2, 4, seed, randomized)


def paper_riemann_state(x, y, gamma: float = GAMMA) -> np.ndarray:
    """Section 6.3 (3): (rho, u, v, p) = (1, 0, -0.3, 1) on [0.5, 1]^2, (2, 0, 0.3, 1) on
    [0, 0.5] x [0.5, 1], (1.0625, 0, 0.8145, 0.4) on [0, 0.5]^2, (0.5313, 0, 0.4276, 0.4) on
    [0.5, 1] x [0, 0.5]; the paper runs to t = 0.3 with dt = 0.001 (uniform grid) or 0.0001
    (randomised grid)."""
    right, up = x >= 0.5, y >= 0.5
    states = ((right & up, (1.0, 0.0, -0.3, 1.0)), (~right & up, (2.0, 0.0, 0.3, 1.0)),
              (~right & ~up, (1.0625, 0.0, 0.8145, 0.4)), (right & ~up, (0.5313, 0.0, 0.4276, 0.4)))
    out = np.zeros((4,) + x.shape)
    for mask, w in states:
        q = conservative(*(np.full(x.shape, c) for c in w), gamma=gamma)
        out[:, mask] = q[:, mask]
    return out


def paper_shock_vortex_grid(n: int = 601, randomized: bool = True, seed: int = 1817):
    """Section 6.1 (3): [-20, 10] x [-15, 15] with n x n grid lines (the paper's 600 x 600
    cells), nine uniform layers at the boundaries, A = 0.2 inside; the state is
    shock_vortex_state with the paper's Mach 3 shock, run to t = 15 with dt = 0.01."""
    return _box_grid(n, (-20.0, -15.0), (10.0, 15.0), 0.2, 9, seed, randomized)


# ----------------------------------------------------------------------------------------
# Three dimensions: arrays are (nk, nj, ni), i fastest; states (5, nk, nj, ni)
# ----------------------------------------------------------------------------------------
def conservative3(rho, u, v, w, p, gamma: float = GAMMA) -> np.ndarray:
    return np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def periodic_cube(n: int, length: float, amp: float, seed: int, nj: int | None = None, nk: int | None = None):
    """ni x nj x nk unique nodes of a periodic box [0, length)^3.  Every node moves along one
    of the three coordinates (chosen by a uniform draw, as the two-dimensional randomisation
    picks one of two) by h 2 amp (r - 1/2).  Returns x, y, z, period (3 x 3)."""
    ni, nj, nk = n, (n if nj is None else nj), (n if nk is None else nk)
    h = (length / ni, length / nj, length / nk)
    k, j, i = np.meshgrid(np.arange(nk, dtype=np.float64), np.arange(nj, dtype=np.float64),
                          np.arange(ni, dtype=np.float64), indexing="ij")
    X = [h[0] * i, h[1] * j, h[2] * k]
    if amp > 0:
        N = ni * nj * nk
        which = np.floor(3.0 * uniform(seed, 0, N, 3)).reshape(nk, nj, ni)
        for c in range(3):
            r = uniform(seed, 0, N, c).reshape(nk, nj, ni)
            X[c] = X[c] + h[c] * 2.0 * amp * (r - 0.5) * (which == c)
    period = ((length, 0.0, 0.0), (0.0, length, 0.0), (0.0, 0.0, length))
    return X[0], X[1], X[2], period


def extrude(x, y, nk: int, dz: float = 1.0):
    """A two-dimensional grid repeated along k with spacing dz: x, y, z of shape (nk, nj, ni)."""
    X = np.broadcast_to(x[None], (nk,) + x.shape).copy()
    Y = np.broadcast_to(y[None], (nk,) + y.shape).copy()
    Z = np.broadcast_to(dz * np.arange(nk, dtype=np.float64)[:, None, None], X.shape).copy()
    return X, Y, Z


def vortex3(x, y, z, center, strength=5.0, free=(1.0, 1.0, 1.0, 0.5, 1.0), period=None, gamma: float = GAMMA):
    """The isentropic vortex about an axis parallel to z through (cx, cy), on a free stream
    (rho, u, v, w, p), modulated along z by a smooth density wave of small amplitude, so the
    state varies in all three directions (a smooth input for parity and order checks)."""
    q2 = isentropic_vortex(x.reshape(-1, x.shape[-1]), y.reshape(-1, y.shape[-1]), center, strength,
                           (free[0], free[1], free[2], free[4]),
                           None if period is None else (period[0][0], period[1][1]), gamma=gamma)
    q2 = q2.reshape((4,) + x.shape)
    rho, u, v = q2[0], q2[1] / q2[0], q2[2] / q2[0]
    p = (gamma - 1.0) * (q2[3] - 0.5 * rho * (u * u + v * v))
    Lz = 2.0 * np.pi if period is None else period[2][2]
    rho = rho * (1.0 + 0.05 * np.sin(2.0 * np.pi * z / Lz))
    return conservative3(rho, u, v, np.full_like(rho, free[3]), p, gamma)


def random_state3(shape, seed: int, rho=(0.8, 1.2), vel=(-0.3, 0.3), p=(0.8, 1.2), gamma: float = GAMMA,
                  block: int = 17) -> np.ndarray:
    """Every node independent (algebraic tests), shape (nk, nj, ni)."""
    n = int(np.prod(shape))
    r = [uniform(seed, block + k, n, 0).reshape(shape) for k in range(5)]
    s = lambda lo_hi, t: lo_hi[0] + (lo_hi[1] - lo_hi[0]) * t
    return conservative3(s(rho, r[0]), s(vel, r[1]), s(vel, r[2]), s(vel, r[3]), s(p, r[4]), gamma)
