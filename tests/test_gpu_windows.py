"""Sliding-window local GLCMs and maps vs the oracle."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
from conftest import to_u32
import featcheck

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sym", [False, True])
def test_windows_counts_and_maps(gctx, sym):
    img = S.smooth(3, 150, 203, 4.0, np.uint8)
    offs = S.CONTENTION_OFFSETS
    c, m = gctx.windows(torch.from_numpy(img).cuda(), 16, 15, 4, offs, flags=1 if sym else 0)
    torch.cuda.synchronize()
    want = oracle.window_glcm(img, 16, offs, 15, 4)
    nwy, nwx = (150 - 15) // 4 + 1, (203 - 15) // 4 + 1
    got = to_u32(c).reshape(nwy * nwx, 4, 16, 16)
    assert np.array_equal(got, want)
    maps = oracle.window_maps(want, symmetric=sym)  # (4, n_win, n_off)
    g = m.cpu().numpy().reshape(4, 4, nwy * nwx).transpose(0, 2, 1).astype(np.float64)
    scale = np.maximum(np.abs(maps), featcheck.map_scale(16)[:, None, None])
    err = np.abs(g - maps) / scale
    assert err.max() <= 1e-5, err.max()


def test_windows_levels_and_u16(gctx):
    img = S.iid(5, 40, 45, np.uint16)
    offs = [(1, 0), (0, -2), (-3, 1)]
    c, _ = gctx.windows(torch.from_numpy(img).cuda(), 32, 9, 3, offs, maps=False)
    torch.cuda.synchronize()
    want = oracle.window_glcm(img, 32, offs, 9, 3)
    assert np.array_equal(to_u32(c).reshape(want.shape), want)


@pytest.mark.parametrize("win, stride, n, sym", [(21, 5, 12, True), (260, 1, 4, False)])
def test_windows_wide_counters(gctx, win, stride, n, sym):
    """Windows with more than 255 pairs per offset (16-bit counters: 21 x 21)
    and more than 65535 (32-bit counters: 260 x 260), a level count that is not
    a power of two, counts and maps against the oracle."""
    side = win + 10 * stride
    img = S.smooth(40 + win, side, side, 3.0, np.uint8)
    offs = [(1, 0), (1, -1)] if win < 100 else [(1, 0)]
    c, m = gctx.windows(torch.from_numpy(img).cuda(), n, win, stride, offs, flags=1 if sym else 0)
    torch.cuda.synchronize()
    want = oracle.window_glcm(img, n, offs, win, stride)
    nw = (side - win) // stride + 1
    got = to_u32(c).reshape(nw * nw, len(offs), n, n)
    assert np.array_equal(got, want)
    maps = oracle.window_maps(want, symmetric=sym)
    g = m.cpu().numpy().reshape(4, len(offs), nw * nw).transpose(0, 2, 1).astype(np.float64)
    scale = np.maximum(np.abs(maps), featcheck.map_scale(n)[:, None, None])
    assert (np.abs(g - maps) / scale).max() <= 1e-5


def test_windows_maps_only(gctx):
    """Maps without counts (the per-window GLCMs never leave shared memory):
    bit-identical to the maps written beside the counts, and within the
    feature tolerance of the oracle."""
    img = S.smooth(11, 96, 131, 2.0, np.uint8)
    offs = S.CONTENTION_OFFSETS
    t = torch.from_numpy(img).cuda()
    c, m_both = gctx.windows(t, 16, 15, 4, offs, flags=1)
    none, m_only = gctx.windows(t, 16, 15, 4, offs, flags=1, counts=False)
    torch.cuda.synchronize()
    assert none is None
    assert torch.equal(m_only, m_both)
    want = oracle.window_glcm(img, 16, offs, 15, 4)
    nwy, nwx = (96 - 15) // 4 + 1, (131 - 15) // 4 + 1
    maps = oracle.window_maps(want, symmetric=True)
    g = m_only.cpu().numpy().reshape(4, 4, nwy * nwx).transpose(0, 2, 1).astype(np.float64)
    scale = np.maximum(np.abs(maps), featcheck.map_scale(16)[:, None, None])
    assert (np.abs(g - maps) / scale).max() <= 1e-5
