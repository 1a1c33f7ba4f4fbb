"""Gray-level histograms (glcm_histogram) vs the oracle, bit-exact.

Contiguous images (the whole grid strides over one span), pitched views with
odd bases and pitches (warps take row segments; bytes before the first and
after the last 16-byte boundary are read one pixel at a time; uint16 rows at
odd addresses are read bytewise), smooth, constant and noise images at every
level count class, host buffers, 1 x 1 and one-row images, and out-of-range
pixels in levels mode."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("kind", ["iid", "smooth", "constant"])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("n", [2, 7, 16, 256])
def test_histogram_contiguous(gctx, kind, dtype, n):
    img = S.image(kind, 11, 1031, 517, dtype, 4.0)
    got = to_u32(gctx.histogram(dev(img), n))
    assert np.array_equal(got, oracle.histogram(img, n))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("x0, w", [(0, 4096), (1, 4095), (3, 100), (5, 9000), (7, 1)])
def test_histogram_pitched_views(gctx, dtype, x0, w):
    """Column slices of a wider tensor: pitch > row bytes, rows starting at
    any element (uint16 rows at odd byte addresses are covered below)."""
    full = S.iid(21, 37, x0 + w + 3, dtype)
    t = dev(full)[:, x0:x0 + w]
    got = to_u32(gctx.histogram(t, 32))
    assert np.array_equal(got, oracle.histogram(full[:, x0:x0 + w], 32))


@pytest.mark.parametrize("odd_pitch", [False, True])
def test_histogram_u16_odd_addresses(gctx, odd_pitch):
    """uint16 rows starting at odd byte addresses, through the raw C ABI."""
    h, w = 29, 301
    rng = np.random.default_rng(5)
    img = rng.integers(0, 65536, size=(h, w)).astype(np.uint16)
    pitch = 2 * w + (3 if odd_pitch else 6)
    raw = np.zeros(1 + pitch * h + 16, dtype=np.uint8)
    for y in range(h):
        raw[1 + y * pitch:1 + y * pitch + 2 * w] = img[y].view(np.uint8)
    draw = torch.from_numpy(raw).cuda()
    hist = torch.empty(64, dtype=torch.int32, device="cuda")
    G.binding.glcm_histogram(gctx.ctx, draw.data_ptr() + 1, w, h, pitch, G.GLCM_U16, 64, 0, hist)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(hist), oracle.histogram(img, 64))


def test_histogram_host_buffers_and_tiny(gctx):
    img = S.smooth(3, 333, 1000, 2.0, np.uint8)
    got = gctx.histogram(img, 16)  # host image, host result
    assert np.array_equal(to_u32(got), oracle.histogram(img, 16))
    for shape in [(1, 1), (1, 999), (999, 1), (2, 15), (3, 16)]:
        im = S.iid(9, shape[0], shape[1], np.uint8)
        assert np.array_equal(to_u32(gctx.histogram(dev(im), 8)), oracle.histogram(im, 8)), shape


def test_histogram_full_size(gctx):
    """A 4096 x 4096 uint8 image of each kind at N = 256 (the contention
    sweep's image size), bit-exact."""
    for kind in S.CONTENTION_KINDS:
        img = S.image(kind, 2, 4096, 4096, np.uint8, 8.0)
        got = to_u32(gctx.histogram(dev(img), 256))
        assert np.array_equal(got, oracle.histogram(img, 256)), kind
        assert int(got.astype(np.int64).sum()) == 4096 * 4096


def test_histogram_levels_mode_range(gctx):
    img = S.iid(4, 64, 640, np.uint8, 0, 8)
    img[10, 100] = 9
    img[33, 5] = 200
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError) as ei:
        gctx.histogram(dev(img), 8, G.GLCM_INPUT_LEVELS, out=out)
    assert ei.value.status == G.binding.GLCM_ERR_RANGE
    want, skipped = oracle.histogram(img, 8, levels_mode=True, return_skipped=True)
    assert skipped == 2 and np.array_equal(to_u32(out), want)
    ok = S.iid(4, 64, 640, np.uint16, 0, 200)
    assert np.array_equal(to_u32(gctx.histogram(dev(ok), 200, G.GLCM_INPUT_LEVELS)),
                          oracle.histogram(ok, 200, levels_mode=True))
