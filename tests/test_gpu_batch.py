"""Multi-block batch (fsp_batch_*) against the oracle's multi-block path: metrics with the
ghost layers, right-hand sides and RK3 steps of every block, on cylinder blocks (uneven
sizes, randomised blocks, slip wall, far field, angular wrap) and on a grid whose second
block is stored rotated behind reversed links."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def F():
    from paper_1810_11103_gb300 import build, fsp
    build.build()
    return fsp


def _small_cylinder():
    blocks, states, free = I.cylinder_blocks(imin=24, imax=48, jmin=16, jmax=32, step=8, cols=4, rows=3,
                                             stretch=1.02, frac_random=0.5)
    return blocks, states, free


def _cfgd(free, scheme=2, prec=0):
    return dict(scheme=scheme, precision=prec, bc_state=np.tile(free, (4, 1)))


def _perturbed(states, seed, amp):
    """Each block's state with its primitive variables perturbed by a relative amp (the
    pressure stays positive)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in states:
        rho = q[0] * (1 + amp * rng.standard_normal(q[0].shape))
        u = q[1] / q[0] + amp * rng.standard_normal(q[0].shape)
        v = q[2] / q[0] + amp * rng.standard_normal(q[0].shape)
        p = 0.4 * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0]) * (1 + amp * rng.standard_normal(q[0].shape))
        out.append(I.conservative(rho, u, v, p))
    return out


def _maxrel(As, Bs):
    scale = max(np.abs(b).max() for b in Bs)
    return max(np.abs(a - b).max() for a, b in zip(As, Bs)) / scale


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_batch_metrics_and_rhs_small_cylinder(F, scheme):
    blocks, states, free = _small_cylinder()
    cfgd = _cfgd(free, scheme)
    Ms = O.mb_metrics(cfgd, blocks)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, states)
    Mg = [m.cpu().numpy() for m in bt.metrics()]
    for a, b in zip(Mg, Ms):
        assert np.abs(a[:4] - b[:4]).max() < TOL * np.abs(b[:4]).max()
        assert np.abs(a[4] - b[4]).max() < TOL * np.abs(b[4]).max()
    # perturb the free stream so the right-hand side is not trivially zero
    qs = _perturbed(states, scheme, 0.05)
    for k, q in enumerate(qs):
        bt.Q[k].copy_(torch.as_tensor(q))
        # both sides take the far-field inflow/outflow decision (the sign of the free
        # stream's normal velocity, zero where it runs tangent to the outer circle) from
        # the same metrics
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    Rg = [r.cpu().numpy() for r in bt.rhs()]
    Ro = O.mb_rhs(cfgd, blocks, Ms, qs)
    assert _maxrel(Rg, Ro) < TOL
    bt.close()


@pytest.mark.parametrize("variant", [0, 3])
def test_batch_rk3_eager_and_graph(F, variant):
    blocks, states, free = _small_cylinder()
    cfgd = _cfgd(free, 3)
    Ms = O.mb_metrics(cfgd, blocks)
    dt = 2e-4   # well inside the CFL limit of the smallest wall cells
    q2 = O.mb_rk3(cfgd, blocks, Ms, states, dt, 2)
    q4 = O.mb_rk3(cfgd, blocks, Ms, states, dt, 4)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, states)
    for k in range(len(blocks)):
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    bt.set_tile_shape(0, variant)
    bt.set_tile_shape(1, variant)
    bt.rk3_step(dt)
    bt.rk3_step(dt)
    torch.cuda.synchronize()
    assert _maxrel([q.cpu().numpy() for q in bt.Q], q2) < TOL
    bt.capture_graph(dt)          # one eager step, then the captured step
    bt.rk3_step(dt)
    torch.cuda.synchronize()
    assert _maxrel([q.cpu().numpy() for q in bt.Q], q4) < TOL
    bt.close()


def test_batch_reversed_links(F):
    x, y, per = I.periodic_square(30, 8.0, 0.2, seed=3, nj=24)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x / 8.0) * np.cos(2 * np.pi * y / 8.0)
    q = I.conservative(rho, 0.6 + 0.1 * np.cos(2 * np.pi * y / 8.0), np.full_like(x, -0.3), rho * 1.1)
    blocks, qs = I.split_blocks(x, y, q, (14,), (), (0, 0, 1, 1), period=((8.0, 0.0), (0.0, 0.0)))
    B = dict(blocks[1])
    B["x"], B["y"] = blocks[1]["x"][::-1, ::-1].copy(), blocks[1]["y"][::-1, ::-1].copy()
    B["bc"] = [5, 5, 1, 1]
    B["links"] = [(0, 0, 1), (0, 1, 1), None, None]
    B["offsets"] = [blocks[1]["offsets"][1], blocks[1]["offsets"][0], None, None]
    A = dict(blocks[0])
    A["links"] = [(1, 0, 1), (1, 1, 1), None, None]
    blocks2 = [A, B]
    qs2 = [qs[0], qs[1][:, ::-1, ::-1].copy()]
    cfgd = dict(scheme=3)
    Ms = O.mb_metrics(cfgd, blocks2)
    Ro = O.mb_rhs(cfgd, blocks2, Ms, qs2)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks2, qs2)
    Mg = [m.cpu().numpy() for m in bt.metrics()]
    assert max(np.abs(a - b).max() for a, b in zip(Mg, Ms)) < TOL * max(np.abs(b).max() for b in Ms)
    assert _maxrel([r.cpu().numpy() for r in bt.rhs()], Ro) < TOL
    bt.close()


def test_batch_full_size_cylinder_float_paths(F):
    # FP32 and mixed at full size, the tuner's marching passes and the tiles, against the
    # oracle on the float-rounded state, under the bounds of the float tests (1e-4, 5e-5).
    # Float round-off grows with max|flux| / max|flux difference|: 7.5 here against 43 on
    # the 256 x 256 vortex (measured 3.8e-5 and 2.2e-5 there), so about 7e-6 and 4e-6 are
    # expected.
    blocks, states, free = I.cylinder_blocks()
    qs = [q.astype(np.float32).astype(np.float64) for q in _perturbed(states, 11, 0.02)]
    cfgd = _cfgd(free, 2)
    Ms = O.mb_metrics(cfgd, blocks)
    Ro = O.mb_rhs(cfgd, blocks, Ms, qs)
    for prec, bound in ((1, 1e-4), (2, 5e-5)):
        bt = F.Batch(F.Config.from_dict(dict(cfgd, precision=prec)), blocks, qs)
        for k in range(len(blocks)):
            bt.M[k].copy_(torch.as_tensor(Ms[k]))
        for v in (3, 2):
            bt.set_tile_shape(0, v)
            bt.set_tile_shape(1, v)
            assert _maxrel([r.double().cpu().numpy() for r in bt.rhs()], Ro) < bound, (prec, v)
        bt.close()


@pytest.mark.parametrize("prec,bound", [(1, 1e-4), (2, 5e-5)])
@pytest.mark.parametrize("scheme", [2, 3])
def test_batch_fp32_paths(F, prec, bound, scheme):
    blocks, states, free = _small_cylinder()
    qs = [q.astype(np.float32).astype(np.float64) for q in _perturbed(states, 7, 0.05)]
    cfgd = _cfgd(free, scheme)
    Ms = O.mb_metrics(cfgd, blocks)
    Ro = O.mb_rhs(cfgd, blocks, Ms, qs)
    bt = F.Batch(F.Config.from_dict(dict(cfgd, precision=prec)), blocks, qs)
    for k in range(len(blocks)):
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    for v in (0, 3):
        bt.set_tile_shape(0, v)
        bt.set_tile_shape(1, v)
        assert _maxrel([r.double().cpu().numpy() for r in bt.rhs()], Ro) < bound, v
    # RK3 stages through the tile and the marching passes agree
    dt = 2e-4
    q1 = []
    for v in (0, 3):
        for k in range(len(blocks)):
            bt.Q[k].copy_(torch.as_tensor(qs[k]))
        bt.set_tile_shape(0, v)
        bt.set_tile_shape(1, v)
        bt.rk3_step(dt)
        q1.append([q.double().cpu().numpy() for q in bt.Q])
    change = [a - b for a, b in zip(q1[0], qs)]
    assert _maxrel([a - b for a, b in zip(q1[1], qs)], change) < 1e-3
    bt.close()


def test_batch_full_size_cylinder(F):
    # the 64-block cylinder workload at full size (5,923,840 nodes), as the bench times it
    blocks, states, free = I.cylinder_blocks()
    qs = _perturbed(states, 11, 0.02)
    cfgd = _cfgd(free, 2)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, qs)
    Mg = [m.cpu().numpy() for m in bt.metrics()]
    Ms = O.mb_metrics(cfgd, blocks)
    assert max(np.abs(a[:4] - b[:4]).max() / np.abs(b[:4]).max() for a, b in zip(Mg, Ms)) < TOL
    Ro = O.mb_rhs(cfgd, blocks, Ms, qs)
    for k in range(len(blocks)):              # identical metrics isolate the right-hand side
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    ref = [r.cpu().numpy() for r in bt.rhs()]
    assert _maxrel(ref, Ro) < TOL
    bt.set_tile_shape(0, 3)                   # marching passes
    bt.set_tile_shape(1, 3)
    assert _maxrel([r.cpu().numpy() for r in bt.rhs()], Ro) < TOL
    bt.close()


@pytest.mark.parametrize("scheme,prec", [(2, 0), (3, 0), (0, 1), (3, 2), (4, 0), (4, 1)])
def test_batch_tile_shapes_agree(F, scheme, prec):
    # every tile shape computes each interface with the same device functions; each kernel
    # instantiation may contract products into FMAs its own way, so FP64 right-hand sides
    # agree to the last bits (1e-13 of the largest value) and float ones to 1e-5
    blocks, states, free = _small_cylinder()
    cfgd = _cfgd(free, scheme, prec)
    qs = _perturbed(states, 3, 0.05)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, qs)
    bt.metrics()
    ref = [r.double().cpu().numpy() for r in bt.rhs()]
    bound = (1e-13 if prec == 0 else 1e-5) * max(np.abs(r).max() for r in ref)
    shapes = set()
    for vx in range(4):          # variant 3: marching warps (xi) and marching CTAs (eta)
        for ve in range(4):
            bt.set_tile_shape(0, vx)
            bt.set_tile_shape(1, ve)
            shapes.add((bt.tile_shape(0), bt.tile_shape(1)))
            got = [r.double().cpu().numpy() for r in bt.rhs()]
            assert max(np.abs(a - b_).max() for a, b_ in zip(got, ref)) <= bound, (vx, ve)
    assert len(shapes) == 16
    with pytest.raises(F.FspError):
        bt.set_tile_shape(1, 4)
    bt.close()


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(1100, 6), (6, 1100), (45, 70)])
def test_batch_marching_segments(F, scheme, shape):
    # lines longer than one marching segment: rows of 1100 nodes (xi: three segments of 384,
    # 384, 332), columns of 1100 nodes (eta: FP64 segments of 126 or 125 rows), partial warps (6 and
    # 45 columns); periodic in both directions, against the oracle and the tile variants
    ni, nj = shape
    x, y, per = I.periodic_square(ni, 10.0, 0.2, seed=5, nj=nj)
    q = I.random_state(x.shape, seed=9)
    cfgd = dict(scheme=scheme, period=per)
    M = O.metrics(cfgd, x, y)
    Ro = O.rhs(cfgd, M, q)
    bt = F.Batch(F.Config.from_dict(cfgd), [dict(x=x, y=y, bc=(0, 0, 0, 0), period=per)], [q])
    bt.M[0].copy_(torch.as_tensor(M))
    bt.set_tile_shape(0, 3)
    bt.set_tile_shape(1, 3)
    got = bt.rhs()[0].cpu().numpy()
    assert np.abs(got - Ro).max() / np.abs(Ro).max() < TOL
    bt.set_tile_shape(0, 0)
    bt.set_tile_shape(1, 0)
    ref = bt.rhs()[0].cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    bt.close()


@pytest.mark.parametrize("shape", [(1100, 6), (6, 1100), (45, 70)])
def test_batch_rk3_marching_line_maxima(F, shape):
    # with the marching eta pass, stages 1 and 2 take the next stage's line maxima from the
    # states they write (per row across the CTAs of a row, per column across the segments of
    # a column); two RK3 steps against the oracle, eagerly and from the captured graph
    ni, nj = shape
    x, y, per = I.periodic_square(ni, 10.0, 0.2, seed=6, nj=nj)
    q = I.random_state(x.shape, seed=10)
    cfgd = dict(scheme=2, period=per)
    M = O.metrics(cfgd, x, y)
    dt = 1e-3
    q2 = O.rk3(cfgd, M, q, dt, 2)
    for graph in (False, True):
        bt = F.Batch(F.Config.from_dict(cfgd), [dict(x=x, y=y, bc=(0, 0, 0, 0), period=per)], [q])
        bt.M[0].copy_(torch.as_tensor(M))
        bt.set_tile_shape(0, 3)
        bt.set_tile_shape(1, 3)
        if graph:
            bt.capture_graph(dt)          # one eager step, then the captured step
        else:
            bt.rk3_step(dt)
        bt.rk3_step(dt)
        torch.cuda.synchronize()
        got = bt.Q[0].cpu().numpy()
        assert np.abs(got - q2).max() / np.abs(q2).max() < TOL, graph
        bt.close()


def test_batch_tune_table(F, tmp_path):
    blocks, states, free = _small_cylinder()
    bt = F.Batch(F.Config.from_dict(_cfgd(free, 2)), blocks, states)
    bt.metrics()
    table = tmp_path / "tiles.txt"
    first = bt.tune(str(table))
    lines = [l for l in table.read_text().splitlines() if l and not l.startswith("#")]
    assert len(lines) == 1
    key, vx, ve = lines[0].split()[:3]
    assert (int(vx), int(ve)) == (first[0][0], first[1][0])
    # a forced shape is replaced by the stored choice, without a new entry
    bt.set_tile_shape(0, (first[0][0] + 1) % 3)
    assert bt.tune(str(table)) == first
    assert len([l for l in table.read_text().splitlines() if l and not l.startswith("#")]) == 1
    # the tuned batch still steps correctly
    Ms = O.mb_metrics(_cfgd(free, 2), blocks)
    for k in range(len(blocks)):
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    q1 = O.mb_rk3(_cfgd(free, 2), blocks, Ms, states, 2e-4, 1)
    bt.capture_graph(2e-4)
    torch.cuda.synchronize()
    assert _maxrel([q.cpu().numpy() for q in bt.Q], q1) < TOL
    bt.close()


def test_batch_flat_state_round_trip(F):
    """The states are views of one buffer: a whole-batch host copy in, one RK3 step, one copy
    out gives the same states as the per-block tensors."""
    blocks, states, free = _small_cylinder()
    cfgd = _cfgd(free, 2)
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, _perturbed(states, 7, 0.01))
    bt.metrics()
    for k, q in enumerate(bt.Q):
        assert q.data_ptr() % 512 == 0 and q.untyped_storage().data_ptr() == bt.Qflat.untyped_storage().data_ptr()
    host = bt.Qflat.cpu().pin_memory()
    bt.Qflat.zero_()
    bt.Qflat.copy_(host, non_blocking=True)
    bt.rk3_step(1e-3)
    out = torch.empty_like(host).pin_memory()
    out.copy_(bt.Qflat, non_blocking=True)
    torch.cuda.synchronize()
    for q in bt.Q:
        off = (q.data_ptr() - bt.Qflat.data_ptr()) // q.element_size()
        assert torch.equal(out[off:off + q.numel()].view(q.shape), q.cpu())
        assert not torch.equal(q.cpu(), host[off:off + q.numel()].view(q.shape))   # the step changed it


def test_batch_rk3_step_host(F):
    """fsp_batch_rk3_step_host equals the device step bit for bit: with the host arrays laid
    out like Qflat (merged copies), pinned or pageable, in place, and with each block in a
    host tensor of its own (one copy per block); device pointers are refused."""
    import ctypes
    blocks, states, free = _small_cylinder()
    cfgd = _cfgd(free, 2)
    qs = _perturbed(states, 5, 0.01)
    dt = 2e-4
    ref = F.Batch(F.Config.from_dict(cfgd), blocks, qs)
    ref.metrics()
    ref.rk3_step(dt)
    want = ref.Qflat.cpu()
    ref.close()
    bt = F.Batch(F.Config.from_dict(cfgd), blocks, qs)
    bt.metrics()
    start = bt.Qflat.cpu()
    for pinned, inplace in ((True, False), (False, False), (True, True)):
        hin = start.clone().pin_memory() if pinned else start.clone()
        hout = hin if inplace else torch.full_like(hin, np.nan)
        bt.Qflat.fill_(np.nan)                                 # the step must start from hin
        bt.rk3_step_host(dt, hin, hout)
        torch.cuda.synchronize()
        assert torch.equal(hout, want), (pinned, inplace)
    # separate host tensors per block: one copy each
    other = F.Batch(F.Config.from_dict(cfgd), blocks, qs)
    sep_in = [q.cpu().clone() for q in other.Q]
    other.close()
    sep_out = [torch.empty_like(q) for q in sep_in]
    tab = lambda ts: (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    rc = F.lib().fsp_batch_rk3_step_host(bt._h, tab(sep_in), tab(sep_out), dt, None)
    assert rc == 0
    torch.cuda.synchronize()
    for q, o in zip(bt.Q, sep_out):
        off = (q.data_ptr() - bt.Qflat.data_ptr()) // q.element_size()
        assert torch.equal(o.view(-1), want[off:off + q.numel()])
    dev = (ctypes.c_void_p * bt.n)(*[q.data_ptr() for q in bt.Q])
    assert F.lib().fsp_batch_rk3_step_host(bt._h, dev, tab(sep_out), dt, None) == 1
    with pytest.raises(ValueError):
        bt.rk3_step_host(dt, bt.Qflat, start)
    bt.close()


def test_batch_full_size_cylinder_rk3(F):
    """One RK3 step of the 64-block cylinder at full size (5,923,840 nodes) as the bench runs it
    end to end: tuned tiles, the captured graph, host copies through fsp_batch_rk3_step_host;
    against the oracle's multi-block step on the same metrics, at the bench's CFL 0.3 step."""
    blocks, states, free = I.cylinder_blocks()
    qs = _perturbed(states, 13, 0.02)
    cfgd = _cfgd(free, 2)
    cfg = F.Config.from_dict(cfgd)
    Ms = O.mb_metrics(cfgd, blocks)
    bt = F.Batch(cfg, blocks, qs)
    for k in range(len(blocks)):
        bt.M[k].copy_(torch.as_tensor(Ms[k]))
    bt.tune()
    dt = min(float(F.cfl_dt(F.Config.from_dict(dict(cfgd, bc=[1 if c == 5 else c for c in b["bc"]])),
                            bt.M[k], bt.Q[k], 0.3).item()) for k, b in enumerate(blocks))
    host = bt.Qflat.cpu().pin_memory()
    bt.capture_graph(dt)                           # an eager step, then the graph
    out = torch.empty_like(host).pin_memory()
    bt.rk3_step_host(dt, host, out)
    torch.cuda.synchronize()
    q1 = O.mb_rk3(cfgd, blocks, Ms, qs, dt, 1)
    got = []
    for q in bt.Q:
        off = (q.data_ptr() - bt.Qflat.data_ptr()) // q.element_size()
        got.append(out[off:off + q.numel()].view(q.shape).numpy())
    assert _maxrel([g - q for g, q in zip(got, qs)], [a - q for a, q in zip(q1, qs)]) < 1e-11
    assert _maxrel(got, q1) < TOL
    bt.close()
