"""The paper's own test problems on the GPU, at the paper's sizes and time steps
(Sections 5.2, 6.2 and 6.3), FP64.

Each case is marched on the GPU and, with the same fixed steps, by the oracle: the states
agree to 1e-10 (relative max-norm), over the paper's whole run where the oracle finishes it in
seconds, else over its first steps.  The GPU then finishes the paper's run, and the result is
checked against what the mathematics fixes:
* Table 4 (Section 5.2): uniform Mach 0.5 flow on the 81 x 81 randomised grid, t = 10,
  dt = 0.01 (1000 steps); L2(v) stays at the printed round-off level.
* Sod (Section 6.2 (1)): 100 nodes on [-5, 5], t = 2, dt = 0.01; density against the exact
  Riemann solution.
* Shu-Osher (Section 6.2 (2)): 400 nodes, t = 1.8, dt = 0.001; density against the same run
  on a grid eight times finer.
* Vortex preservation (Section 6.3 (1)): the 81 x 81 periodic grids (uniform and randomised,
  A = 0.45), t = 16, dt = 0.01; after one period v along the centre line against the exact
  (initial) profile.
* Cylinder at Mach 4 (Section 6.3 (2)): the 121 x 41 grids, dt = 0.001 after a start at half
  that step; the stagnation pressure of the converged flow against Rayleigh's pitot formula.
* Riemann problem (Section 6.3 (3)): 401 x 401 grid lines, t = 0.3, dt = 0.001 (uniform) and
  0.0001 (randomised); the two grids' densities against each other.
* Shock-vortex interaction (Section 6.3 (4)): 601 x 601 grid lines, Mach 3 shock, t = 15,
  dt = 0.01 on the randomised grid; the state stays physical."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TOL = 1e-10


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


class Run:
    """A block on the GPU: metrics from the coordinates, the state marched in place."""

    def __init__(self, F, cfgd, x, y, q):
        self.F, self.cfgd = F, cfgd
        self.cfg = F.Config.from_dict(cfgd)
        self.M = F.metrics(self.cfg, torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"))
        self.Q = torch.as_tensor(np.ascontiguousarray(q), device="cuda")
        self.ws = F.workspace(self.cfg, self.Q)

    def march(self, dt, nsteps):
        for _ in range(nsteps):
            self.F.rk3_step(self.cfg, self.M, self.Q, dt, ws=self.ws)
        torch.cuda.synchronize()
        return self.Q.cpu().numpy()


def _parity(F, cfgd, x, y, q, dt, nsteps):
    """GPU and oracle march the same steps; returns the GPU run (state after nsteps)."""
    run = Run(F, cfgd, x, y, q)
    qg = run.march(dt, nsteps)
    qo = O.rk3(cfgd, O.metrics(cfgd, x, y), q, dt, nsteps)
    assert _rel(qg, qo) <= TOL, _rel(qg, qo)
    return run


def _table4():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table4.csv")
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    return [float(r.split(",")[1]) for r in rows]


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_table4_free_stream_full_run(F, scheme):
    x, y = I.paper_random_grid(81, 81, 16.0, 0.45, seed=1810)
    cfgd = dict(scheme=scheme, bc=(1, 1, 1, 1))
    q = I.uniform_state(x.shape, 1.0, 0.5, 0.0, 1.0 / GAMMA)
    run = _parity(F, cfgd, x, y, q, 0.01, 50)
    qf = run.march(0.01, 950)                    # t = 10
    v = qf[2] / qf[0]
    l2 = math.sqrt(float((v * v).mean()))
    printed = _table4()[scheme]
    print(f"table4 scheme {scheme}: L2(v) {l2:.3e} (printed {printed:.3e})")
    # round-off: the printed 1.5e-15 .. 2.5e-15 depend on the order of the paper's own
    # arithmetic; the same magnitude is required
    assert l2 < 4.0 * printed, (l2, printed)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_paper_sod(F, scheme):
    x, y, q, per = I.paper_sod(100)
    cfgd = dict(scheme=scheme, bc=(1, 1, 0, 0), period=per)
    run = _parity(F, cfgd, x, y, q, 0.01, 200)   # the whole run, t = 2
    qf = run.Q.cpu().numpy()
    WL, WR = np.array([0.125, 0.0, 0.1]), np.array([1.0, 0.0, 1.0])
    ex = O.riemann_exact(GAMMA, WL, WR, 0.0, 2.0, x[0])
    l1 = float(np.abs(qf[0, 0] - ex[:, 0]).mean())
    print(f"paper Sod scheme {scheme}: density L1 against the exact solution {l1:.3e}")
    assert l1 < 1e-2, l1
    # mass is conserved while no wave has reached the ends
    assert abs(qf[0].sum() - q[0].sum()) < 1e-12 * q[0].sum()


@pytest.mark.parametrize("scheme", [1, 2])
def test_shu_osher(F, scheme):
    x, y, q, per = I.shu_osher(400)
    cfgd = dict(scheme=scheme, bc=(1, 1, 0, 0), period=per)
    run = _parity(F, cfgd, x, y, q, 0.001, 1800)  # the whole run, t = 1.8
    qf = run.Q.cpu().numpy()
    xf, yf, qf8, perf = I.shu_osher(8 * 399 + 1)  # nested: every 8th fine node is a coarse one
    fine = Run(F, dict(cfgd, period=perf), xf, yf, qf8).march(0.001 / 8, 8 * 1800)
    assert np.array_equal(xf[0, ::8], x[0])
    d = np.abs(qf[0, 0] - fine[0, 0, ::8])
    print(f"Shu-Osher scheme {scheme}: density L1 / Linf against the 3193-node run {d.mean():.3e} / {d.max():.3e}")
    assert float(d.mean()) < 0.06, float(d.mean())
    assert qf[0].min() > 0.5 and qf[0].max() < 5.0


@pytest.mark.parametrize("randomized", [False, True])
def test_paper_vortex_one_period(F, randomized):
    x, y, per = I.paper_vortex_grid(81, randomized=randomized)
    q = I.paper_vortex_state(x, y, per)
    cfgd = dict(scheme=2, period=per)
    run = _parity(F, cfgd, x, y, q, 0.01, 40)
    qf = run.march(0.01, 1560)                   # t = 16: one period
    j = 40                                       # the grid line j = Jmax/2 + 1 (1-based) through the centre
    v_num, v_ex = qf[2, j] / qf[0, j], q[2, j] / q[0, j]
    err = float(np.abs(v_num - v_ex).max())
    print(f"vortex randomized={randomized}: max |v - v_exact| on the centre line after one period {err:.3e}")
    # the vortex's peak speed is 0.3 e^{alpha} ~ 0.37 (r = 1); after one period on h = 0.2
    assert err < (0.05 if randomized else 0.03), err


def _pitot(mach, p1, g=GAMMA):
    """Stagnation pressure behind a normal shock (Rayleigh's pitot formula)."""
    m2 = mach * mach
    return p1 * ((g + 1) * m2 / 2) ** (g / (g - 1)) * ((g + 1) / (2 * g * m2 - (g - 1))) ** (1 / (g - 1))


@pytest.mark.parametrize("randomized", [False, True])
def test_paper_cylinder_stagnation_pressure(F, randomized):
    x, y, bc, st = I.paper_cylinder(randomized=randomized)
    cfgd = dict(scheme=2, bc=bc, bc_state=st)
    q = np.broadcast_to(st[0][:, None, None], (4,) + x.shape).copy()
    # the impulsive start (the free stream against the wall) blows up at the paper's step:
    # half of it until t = 0.1, the paper's dt = 0.001 after that (CFL about 0.4 then)
    run = _parity(F, cfgd, x, y, q, 0.0005, 40)
    run.march(0.0005, 160)
    qf = run.march(0.001, 19900)                 # t = 20: the bow shock has settled
    rho, mu, mv, E = qf[:, 0, :]
    p = (GAMMA - 1) * (E - 0.5 * (mu * mu + mv * mv) / rho)
    p_stag = float(p[x.shape[1] // 2])           # the wall node on the stagnation line
    ref = _pitot(4.0, 1.0 / GAMMA)
    print(f"cylinder randomized={randomized}: stagnation pressure {p_stag:.4f}, pitot {ref:.4f}")
    assert abs(p_stag / ref - 1.0) < 0.03, (p_stag, ref)
    qm = run.march(0.001, 1000)
    assert _rel(qm, qf) < 1e-3                   # steady


def test_paper_riemann(F):
    out = {}
    for randomized, dt, n in ((False, 1e-3, 300), (True, 1e-4, 3000)):
        x, y = I.paper_riemann_grid(401, randomized=randomized)
        q = I.paper_riemann_state(x, y)
        cfgd = dict(scheme=2, bc=(1, 1, 1, 1))
        run = _parity(F, cfgd, x, y, q, dt, 4)
        out[randomized] = run.march(dt, n - 4)      # t = 0.3
        assert out[randomized][0].min() > 0.2 and out[randomized][0].max() < 3.0
    # the randomised grid moves nodes by up to 0.2 h: the solutions agree to the scheme's
    # resolution of the slip lines and shocks
    d = float(np.abs(out[True][0] - out[False][0]).mean())
    print(f"Riemann 401: density range {out[False][0].min():.4f}..{out[False][0].max():.4f}, "
          f"mean |randomised - uniform| {d:.3e}")
    assert d < 0.02


def test_paper_shock_vortex(F):
    x, y = I.paper_shock_vortex_grid(601, randomized=True)
    q = I.shock_vortex_state(x, y, mach=3.0)
    bc, st = I.shock_vortex_bc(mach=3.0)
    cfgd = dict(scheme=2, bc=bc, bc_state=st)
    run = _parity(F, cfgd, x, y, q, 0.01, 2)
    qf = run.march(0.01, 1498)                   # t = 15
    rho = qf[0]
    p = (GAMMA - 1) * (qf[3] - 0.5 * (qf[1] ** 2 + qf[2] ** 2) / rho)
    print(f"shock-vortex 601 Mach 3: density {rho.min():.4f}..{rho.max():.4f}, pressure {p.min():.4f}..{p.max():.4f}")
    assert np.isfinite(qf).all() and rho.min() > 0 and p.min() > 0
