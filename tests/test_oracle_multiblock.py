"""Pins of the oracle's multi-block path (CPU): cutting one grid into linked blocks must
reproduce the single-block metrics (ghost layers included) and, where the per-block-line
maxima equal the per-line ones, the single-block right-hand side; a block stored rotated
by 180 degrees behind a reversed link gives the same values; uniform flow is preserved."""
import numpy as np
import pytest

import oracle as O
from paper_1810_11103_gb300 import inputs as I

G = O.G


def _slices(isplit, jsplit, ni, nj):
    ic = [0] + list(isplit) + [ni]
    jc = [0] + list(jsplit) + [nj]
    out = []
    for b in range(len(jc) - 1):
        for a in range(len(ic) - 1):
            out.append((slice(jc[b], jc[b + 1]), slice(ic[a], ic[a + 1])))
    return out


@pytest.mark.parametrize("scheme", [0, 3])
def test_cut_periodic_grid_reproduces_metrics(scheme):
    ni, nj = 40, 36
    x, y, per = I.periodic_square(ni, 8.0, 0.2, seed=21, nj=nj)
    cfg = dict(scheme=scheme, period=per)
    M1 = O.metrics(cfg, x, y)
    isp, jsp = (13, 27), (11, 20)
    blocks, _ = I.split_blocks(x, y, None, isp, jsp, (0, 0, 0, 0), period=per)
    Ms = O.mb_metrics(cfg, blocks)
    for (sj, si), M in zip(_slices(isp, jsp, ni, nj), Ms):
        # the block's extended range, ghosts included, is a window of the periodic field
        jj = np.arange(sj.start - G, sj.stop + G) % nj
        ii = np.arange(si.start - G, si.stop + G) % ni
        ref = M1[:, G:-G, G:-G][:, jj][:, :, ii]
        assert np.abs(M - ref).max() < 1e-13


def test_cut_grid_with_physical_faces_reproduces_metrics():
    n = 30
    x, y = I.riemann_grid(n, 0.3, 5)
    cfg = dict(scheme=2, bc=(1, 1, 1, 1))
    M1 = O.metrics(cfg, x, y)
    isp, jsp = (12,), (15,)
    blocks, _ = I.split_blocks(x, y, None, isp, jsp, (1, 1, 1, 1))
    Ms = O.mb_metrics(cfg, blocks)
    for (sj, si), M in zip(_slices(isp, jsp, n, n), Ms):
        ref = M1[:, sj.start:sj.stop + 2 * G, si.start:si.stop + 2 * G]
        assert np.abs(M - ref).max() < 1e-13


def _entropy_wave(x, y, u=0.7, v=-0.4):
    # density varies, velocity and temperature do not: |U^| + c|k^| is uniform on an affine
    # grid, so per-block-line and per-line maxima agree
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x / 8.0) * np.cos(2 * np.pi * y / 8.0)
    return I.conservative(rho, np.full_like(x, u), np.full_like(x, v), rho * 1.0)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_cut_grid_reproduces_rhs(scheme):
    ni, nj = 32, 28
    x, y, per = I.periodic_square(ni, 8.0, 0.0, seed=0, nj=nj)
    q = _entropy_wave(x, y)
    cfg = dict(scheme=scheme, period=per)
    R1 = O.rhs(cfg, O.metrics(cfg, x, y), q)
    isp, jsp = (9, 20), (14,)
    blocks, qs = I.split_blocks(x, y, q, isp, jsp, (0, 0, 0, 0), period=per)
    Rs = O.mb_rhs(cfg, blocks, O.mb_metrics(cfg, blocks), qs)
    for (sj, si), R in zip(_slices(isp, jsp, ni, nj), Rs):
        assert np.abs(R - R1[:, sj, si]).max() < 1e-12 * np.abs(R1).max()


def _rot180(b):
    r = dict(b)
    r["x"], r["y"] = b["x"][::-1, ::-1].copy(), b["y"][::-1, ::-1].copy()
    r["bc"] = [b["bc"][1], b["bc"][0], b["bc"][3], b["bc"][2]]
    r["links"] = [b["links"][1], b["links"][0], b["links"][3], b["links"][2]]
    r["offsets"] = [b["offsets"][1], b["offsets"][0], b["offsets"][3], b["offsets"][2]]
    return r


def _rotated_pair(amp):
    ni, nj = 30, 24
    x, y, per = I.periodic_square(ni, 8.0, amp, seed=3, nj=nj)
    q = _entropy_wave(x, y)
    cfg = dict(scheme=3, period=((8.0, 0.0), (0.0, 0.0)), bc=(0, 0, 1, 1))
    # two blocks side by side, the second stored rotated by 180 degrees: A's i-max meets
    # B's stored i-max and the wrap joins their i-min faces, both reversed
    blocks, qs = I.split_blocks(x, y, q, (14,), (), (0, 0, 1, 1), period=((8.0, 0.0), (0.0, 0.0)))
    A, B = blocks[0], _rot180(blocks[1])
    A["links"] = [(1, 0, 1), (1, 1, 1), None, None]
    B["links"] = [(0, 0, 1), (0, 1, 1), None, None]
    return cfg, x, y, q, A, B, [qs[0], qs[1][:, ::-1, ::-1].copy()]


def test_reversed_link_metrics_on_randomised_grid():
    cfg, x, y, q, A, B, _ = _rotated_pair(0.2)
    M1 = O.metrics(cfg, x, y)
    Ms = O.mb_metrics(cfg, [A, B])
    assert np.abs(Ms[0] - M1[:, :, :14 + 2 * G]).max() < 1e-13
    # rotating the indices by 180 degrees reverses both index directions: the metrics of
    # the rotated block are the negated rotated metrics, J^-1 unchanged
    refB = M1[:, :, 14:][:, ::-1, ::-1].copy()
    refB[:4] *= -1
    assert np.abs(Ms[1] - refB).max() < 1e-13


def test_reversed_link_rhs():
    cfg, x, y, q, A, B, qs = _rotated_pair(0.0)
    R1 = O.rhs(cfg, O.metrics(cfg, x, y), q)
    Rs = O.mb_rhs(cfg, [A, B], O.mb_metrics(cfg, [A, B]), qs)
    tol = 1e-12 * np.abs(R1).max()
    assert np.abs(Rs[0] - R1[:, :, :14]).max() < tol
    assert np.abs(Rs[1][:, ::-1, ::-1] - R1[:, :, 14:]).max() < tol


def test_multiblock_free_stream():
    x, y, per = I.periodic_square(36, 8.0, 0.2, seed=9)
    q = I.uniform_state(x.shape, 1.0, 1.0, 0.5, 1.0)
    cfg = dict(scheme=2, period=per)
    blocks, qs = I.split_blocks(x, y, q, (10, 23), (17,), (0, 0, 0, 0), period=per)
    Rs = O.mb_rhs(cfg, blocks, O.mb_metrics(cfg, blocks), qs)
    assert max(np.abs(R).max() for R in Rs) < 2e-12


def test_small_cylinder_blocks_are_valid():
    blocks, states, free = I.cylinder_blocks(imin=16, imax=32, jmin=16, jmax=24, step=8, cols=4, rows=3,
                                             stretch=1.02)
    assert len(blocks) == 12
    cfg = dict(scheme=2, bc_state=np.tile(free, (4, 1)))
    Ms = O.mb_metrics(cfg, blocks)
    for M in Ms:
        assert (M[4, G:-G, G:-G] > 0).all()   # right-handed, no folded cells
    Rs = O.mb_rhs(cfg, blocks, Ms, states)
    assert all(np.isfinite(R).all() for R in Rs)
