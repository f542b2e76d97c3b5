"""The three-dimensional CUDA path (fsp3_*) against the oracle's three-dimensional path,
element by element on the same seeded inputs.  FP64 bar as in two dimensions: relative
max-norm <= 1e-12 for metrics (the nine direction planes against their common maximum, J^-1
against its own), right-hand sides and RK3 states; line maxima to 1e-13.  Extents are chosen
so that the tiles of every direction end ragged (30 output nodes per tile line for the
one-midpoint schemes, 29 for the two-midpoint ones; 8 xi lines and 16 eta or zeta lines per
tile)."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12
G = 4


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _case(shape=(40, 35, 33), seed=5, bc=(0,) * 6, smooth=True):
    ni, nj, nk = shape
    x, y, z, per = I.periodic_cube(ni, 8.0, 0.2, seed=seed, nj=nj, nk=nk)
    if smooth:
        q = I.vortex3(x, y, z, (4.0, 4.0), strength=4.0, free=(1.0, 0.7, -0.4, 0.3, 1.0), period=per)
    else:
        q = I.random_state3(x.shape, seed=seed + 1)
    return x, y, z, per, q


def _metrics(F, cfgd, blk, x, y, z):
    """Metrics parity.  Each metric is a difference of products of a coordinate (up to X in
    size) and a coordinate difference (up to D, the largest spacing), so each side rounds at a
    few tens of eps X D; J^-1 multiplies them by one more difference: eps X D^2.  These
    absolute floors matter only where one spacing is far below the others (a long thin
    block), where the small metrics' own scale sits below them."""
    cfg = F.Config.from_dict(cfgd)
    M_o = O.metrics3(cfgd, x, y, z)
    M_g = _host(F.metrics3(cfg, blk, _dev(x), _dev(y), _dev(z)))
    X = max(np.abs(c).max() for c in (x, y, z))
    D = max(np.abs(np.diff(c, axis=a)).max() for c in (x, y, z) for a in range(3) if c.shape[a] > 1)
    floor = 64 * np.finfo(np.float64).eps * X * D
    assert np.abs(M_g[:9] - M_o[:9]).max() < TOL * np.abs(M_o[:9]).max() + floor
    assert np.abs(M_g[9] - M_o[9]).max() < TOL * np.abs(M_o[9]).max() + floor * D
    return M_o


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_metrics_and_rhs_parity_ragged_tiles(F, scheme):
    x, y, z, per, q = _case()
    cfgd = dict(scheme=scheme, period=per, bc=(0,) * 6)
    blk = F.block3_of(_dev(x), (0,) * 6, per)
    M = _metrics(F, cfgd, blk, x, y, z)
    R_o = O.rhs3(cfgd, M, q)
    R_g = _host(F.rhs3(F.Config.from_dict(cfgd), blk, _dev(M), _dev(q)))
    assert _rel(R_g, R_o) < TOL, _rel(R_g, R_o)


@pytest.mark.parametrize("scheme", [0, 3, 4])
def test_rhs_parity_random_state_and_transmissive_faces(F, scheme):
    """Every node independent (the weights far from linear), with transmissive faces in i and k."""
    bc = (1, 1, 0, 0, 1, 1)
    x, y, z, per, q = _case((36, 20, 30), seed=9, smooth=False)
    cfgd = dict(scheme=scheme, period=per, bc=bc)
    blk = F.block3_of(_dev(x), bc, per)
    M = _metrics(F, cfgd, blk, x, y, z)
    R_o = O.rhs3(cfgd, M, q)
    R_g = _host(F.rhs3(F.Config.from_dict(cfgd), blk, _dev(M), _dev(q)))
    assert _rel(R_g, R_o) < TOL, _rel(R_g, R_o)


def test_line_maxima_parity(F):
    x, y, z, per, q = _case((40, 35, 33))
    cfgd = dict(scheme=2, period=per, bc=(0,) * 6)
    blk = F.block3_of(_dev(x), (0,) * 6, per)
    M = O.metrics3(cfgd, x, y, z)
    lam = [l.cpu().numpy() for l in F.line_lambda3(F.Config.from_dict(cfgd), blk, _dev(M), _dev(q))]
    for d in range(3):
        ref = O.lambda3(cfgd, M, q, d) / 1.1
        assert np.abs(lam[d] - ref).max() < 1e-13 * np.abs(ref).max(), d


@pytest.mark.parametrize("scheme", [1, 2])
def test_rk3_parity(F, scheme):
    x, y, z, per, q = _case((34, 31, 17), seed=11)
    cfgd = dict(scheme=scheme, period=per, bc=(0,) * 6)
    cfg = F.Config.from_dict(cfgd)
    blk = F.block3_of(_dev(x), (0,) * 6, per)
    M = O.metrics3(cfgd, x, y, z)
    dt = 0.02
    q_o = O.rk3_3(cfgd, M, q, dt, 2)
    Q, Md = _dev(q), _dev(M)
    ws = F.workspace3(cfg, blk)
    for _ in range(2):
        F.rk3_step3(cfg, blk, Md, Q, dt, ws=ws)
    assert _rel(_host(Q), q_o) < TOL


def test_free_stream_on_randomised_cube(F):
    x, y, z, per = I.periodic_cube(48, 6.0, 0.2, seed=5, nj=40, nk=36)
    q0 = np.array([1.0, 0.5, 0.3, -0.2, 2.5])
    for scheme in range(5):
        cfgd = dict(scheme=scheme, period=per, bc=(0,) * 6)
        cfg = F.Config.from_dict(cfgd)
        blk = F.block3_of(_dev(x), (0,) * 6, per)
        Mg = F.metrics3(cfg, blk, _dev(x), _dev(y), _dev(z))
        Q = _dev(q0[:, None, None, None] * np.ones((5,) + x.shape))
        assert float(F.rhs3(cfg, blk, Mg, Q).abs().max()) < 1e-12, scheme


def test_refusals(F):
    x, y, z, per, q = _case((20, 16, 14))
    blk = F.block3_of(_dev(x), (0,) * 6, per)
    for bad, code in ((dict(scheme=2, precision=1), 2), (dict(scheme=2, weights=1), 2), (dict(scheme=7), 1)):
        with pytest.raises(F.FspError) as e:
            F.workspace3(F.Config.from_dict(bad), blk)
        assert e.value.code == code, bad
    cfg = F.Config.from_dict(dict(scheme=2))
    for bc, code in (((2, 2, 0, 0, 0, 0), 2), ((0, 1, 0, 0, 0, 0), 1)):
        with pytest.raises(F.FspError) as e:
            F.workspace3(cfg, F.block3_of(_dev(x), bc, per))
        assert e.value.code == code, bc
    # a non-periodic direction needs 13 nodes (the reflected ghost coordinates)
    xs, ys, zs, pers, _ = _case((20, 16, 12))
    with pytest.raises(F.FspError):
        F.workspace3(cfg, F.block3_of(_dev(xs), (0, 0, 0, 0, 1, 1), pers))


@pytest.mark.parametrize("shape", [(1500, 13, 14), (13, 1500, 14), (14, 13, 1500)])
def test_rhs_parity_long_thin_blocks(F, shape):
    """One long direction of 1500 nodes (50 tiles of 30 output nodes, the last ragged) and two
    short transmissive ones (13 and 14 nodes: partial tiles of 8 lines, reflected ghost
    coordinates); a random state, so every weight is far from linear."""
    ni, nj, nk = shape
    x, y, z, per = I.periodic_cube(ni, 8.0, 0.2, seed=3, nj=nj, nk=nk)
    longest = int(np.argmax(shape))
    bc = tuple(0 if a // 2 == longest else 1 for a in range(6))
    q = I.random_state3(x.shape, seed=4)
    cfgd = dict(scheme=2, period=per, bc=bc)
    blk = F.block3_of(_dev(x), bc, per)
    M = _metrics(F, cfgd, blk, x, y, z)
    R_o = O.rhs3(cfgd, M, q)
    R_g = _host(F.rhs3(F.Config.from_dict(cfgd), blk, _dev(M), _dev(q)))
    assert _rel(R_g, R_o) < TOL, _rel(R_g, R_o)


@pytest.mark.parametrize("nk", [1, 2])
def test_single_layer_blocks_reduce_to_two_dimensions(F, nk):
    """The degenerate case of a block one or two nodes deep, periodic in k: a two-dimensional
    grid extruded along k with a state independent of k.  The three-dimensional kernels equal
    the oracle, and their flux differences equal the two-dimensional kernels' (a separate code
    path) on the same grid; the w equation stays at round-off."""
    x, y, per = I.periodic_square(45, 8.0, 0.2, seed=21, nj=37)
    q2 = I.isentropic_vortex(x, y, (4.0, 4.0), strength=5.0, free=(1.0, 1.0, 0.5, 1.0), period=(8.0, 8.0))
    X, Y, Z = I.extrude(x, y, nk)
    per3 = ((8.0, 0.0, 0.0), (0.0, 8.0, 0.0), (0.0, 0.0, float(nk)))
    Q3 = np.stack([q2[0], q2[1], q2[2], 0.0 * q2[0], q2[3]])[:, None].repeat(nk, axis=1)
    c3 = dict(scheme=2, period=per3, bc=(0,) * 6)
    blk = F.block3_of(_dev(X), (0,) * 6, per3)
    M3 = _metrics(F, c3, blk, X, Y, Z)
    R3 = _host(F.rhs3(F.Config.from_dict(c3), blk, _dev(M3), _dev(Q3)))
    assert _rel(R3, O.rhs3(c3, M3, Q3)) < TOL
    c2 = dict(scheme=2, period=per)
    M2 = _host(F.metrics(F.Config.from_dict(c2), _dev(x), _dev(y)))
    R2 = _host(F.rhs(F.Config.from_dict(c2), _dev(M2), _dev(q2)))
    D3 = R3 * M3[9, G:-G, G:-G, G:-G][None]
    D2 = R2 * M2[4, G:-G, G:-G][None]
    scale = np.abs(D2).max()
    for v3, v2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
        assert np.abs(D3[v3] - D2[v2][None]).max() < 1e-12 * scale, v3
    assert np.abs(D3[3]).max() < 1e-14 * scale
