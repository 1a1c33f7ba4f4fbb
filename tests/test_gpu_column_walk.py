"""The column-walk vote kernel (offsets (D, 0), (D, -D), (0, -D), (-D, -D)
and their opposites at chessboard distance D = 1 .. 4, N a power of two up
to 32, or 256) against the oracle, bit for bit.

It is the default path for those offsets, so these cases aim at what is
special to it: every N and pixel type (joint codes for N <= 8, pairs of
offsets for N = 16, 16-bit halves for N = 32), offsets and their opposites
(counted once, written as counts and transposes), subsets of the four
directions, repeats and other distances beside them (which go to the
general kernel), widths around the 512-byte strips, one-row and one-column
images, pitched views, host images in row stripes (bands whose halo row
lies in the previous stripe), batches mixing both kernels, and a
configured tile height."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32

pytestmark = pytest.mark.gpu

C4 = S.CONTENTION_OFFSETS
OPPOSITE = [(-1, 0), (-1, 1), (0, 1), (1, 1)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(ctx, img, n, offs, flags=0):
    c = ctx.compute(dev(img), n, offs, flags)
    torch.cuda.synchronize()
    return to_u32(c)


def _img(kind, seed, h, w, dt):
    return S.image(kind, seed, h, w, dt, sigma=6.0)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("kind", ["iid", "smooth", "constant"])
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 256])
def test_every_level_count_and_kind(gctx, n, kind, dt):
    img = _img(kind, 100 + n, 300, 1100, dt)
    assert np.array_equal(run(gctx, img, n, C4), oracle.glcm(img, n, C4))


@pytest.mark.parametrize("n", [4, 8, 16, 32, 256])
@pytest.mark.parametrize("offs", [
    [(1, 0)],
    [(0, -1), (1, -1)],
    [(-1, -1), (1, 0), (0, -1)],
    OPPOSITE,
    [(1, 0), (-1, 0), (0, -1), (0, 1)],
    C4 + OPPOSITE,
    [(1, 0), (1, 0), (0, -1)],
    [(1, 0), (2, 0), (0, -1), (-2, -2), (1, 1), (0, -4)],
], ids=["right", "up-pair", "three", "opposites", "both-ways", "all-eight", "repeat", "mixed-distances"])
def test_offset_sets(gctx, n, offs):
    for dt in (np.uint8, np.uint16):
        img = _img("smooth", 7 * n + len(offs), 190, 777, dt)
        img[:, 400:] = _img("iid", 8 * n, 190, 377, dt)
        assert np.array_equal(run(gctx, img, n, offs), oracle.glcm(img, n, offs)), (dt, offs)


@pytest.mark.parametrize("h,w", [(1, 1), (1, 17), (2, 1), (3, 5), (17, 16), (64, 511), (65, 512), (66, 513),
                                 (9, 1024), (33, 1537), (200, 4097)])
@pytest.mark.parametrize("n", [8, 32, 256])
def test_shapes_around_strips(gctx, h, w, n):
    for dt in (np.uint8, np.uint16):
        img = _img("iid", h * 7919 + w, h, w, dt)
        offs = C4 + [(-1, 0)]
        assert np.array_equal(run(gctx, img, n, offs), oracle.glcm(img, n, offs)), dt


def test_pitched_views(gctx):
    base = _img("smooth", 31, 300, 2048, np.uint8)
    t = torch.from_numpy(base).cuda()
    for x0, x1 in [(0, 1000), (16, 1530), (3, 700)]:  # 16-byte aligned starts take the column walk
        c = gctx.compute(t[:, x0:x1], 16, C4)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(c), oracle.glcm(np.ascontiguousarray(base[:, x0:x1]), 16, C4)), (x0, x1)


def test_host_image_in_stripes(gctx):
    img = _img("smooth", 41, 3000, 2000, np.uint8)
    img[1500:] = _img("iid", 42, 1500, 2000, np.uint8)
    for n in (8, 32, 256):
        c = gctx.compute(img, n, C4 + OPPOSITE[:1])
        assert np.array_equal(to_u32(c), oracle.glcm(img, n, C4 + OPPOSITE[:1])), n


def test_batch_mixing_both_kernels(gctx):
    specs = [("iid", 300, 700, np.uint8, 8, C4), ("smooth", 257, 1300, np.uint16, 32, C4),
             ("constant", 90, 90, np.uint8, 16, OPPOSITE), ("iid", 128, 640, np.uint8, 256, C4),
             ("smooth", 200, 333, np.uint8, 4, [(1, 0), (3, -3)]), ("iid", 64, 1024, np.uint16, 2, C4),
             ("smooth", 120, 900, np.uint8, 10, C4)]
    imgs, jobs = [], []
    for k, (kind, h, w, dt, n, offs) in enumerate(specs):
        im = _img(kind, 500 + k, h, w, dt)
        imgs.append(im)
        jobs.append(dict(image=dev(im), levels=n, offsets=offs, flags=G.GLCM_SYMMETRIC, features=True))
    prepared = gctx.prepare(jobs)
    for rep in range(3):  # the direct run, then replays of the captured graph
        for c, _, _ in prepared.outs:
            c.fill_(-1)
        res = gctx.run(prepared)
        torch.cuda.synchronize()
        for im, (_, _, _, _, n, offs), (c, _, _) in zip(imgs, specs, res):
            assert np.array_equal(to_u32(c), oracle.glcm(im, n, offs)), (n, offs, rep)


def test_n256_counts_at_a_misaligned_address_take_the_general_kernel(gctx):
    """N = 256 merges by 16-byte bulk reductions into the output rows; counts
    that do not start on 16 bytes must still come out exact (general kernel)."""
    img = _img("iid", 51, 300, 1000, np.uint8)
    flat = torch.empty(4 * 256 * 256 + 1, dtype=torch.int32, device="cuda")
    out = flat[1:].view(4, 256, 256)
    gctx.compute(dev(img), 256, C4, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(out), oracle.glcm(img, 256, C4))


def test_n256_all_in_one_bin_and_both_halves():
    """A constant image (every vote of an offset in one bin, 16.7 M of them in
    one half's counter), and a two-level image whose rows fall in both halves."""
    with G.Context(0, hbm_budget_bytes=1 << 30) as ctx:
        for img in (np.full((4096, 4096), 200, np.uint8),
                    np.where(_img("smooth", 52, 1024, 2048, np.uint8) > 128, 250, 3).astype(np.uint8)):
            assert np.array_equal(run(ctx, img, 256, C4 + OPPOSITE), oracle.glcm(img, 256, C4 + OPPOSITE))


@pytest.mark.parametrize("band", [8, 100, 1024])
def test_configured_tile_height_and_general_agree(band):
    n, offs = 32, C4
    img = np.full((4100, 512), 77, np.uint8)  # every vote of an offset in one bin
    img[2000:2100] = _img("iid", 9, 100, 512, np.uint8)
    want = oracle.glcm(img, n, offs)
    with G.Context(0, hbm_budget_bytes=1 << 30) as ctx:
        G.glcm_set_vote_config(ctx.ctx, n, len(offs), G.GLCM_U8, 512, 5, 4, band)
        assert np.array_equal(run(ctx, img, n, offs), want)
        G.glcm_set_vote_config(ctx.ctx, n, len(offs), G.GLCM_U8, 512, 3, 1, 0)  # the general kernel
        assert np.array_equal(run(ctx, img, n, offs), want)


@pytest.mark.parametrize("n", [4, 8, 16, 32, 256])
@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_rows_at_any_byte_address(gctx, n, dt):
    """Contiguous images of odd widths (every row at a different alignment, the
    last row ending short of a 16-byte block) and views starting at odd
    columns: the column walk realigns its 16-byte loads."""
    for h, w in [(70, 17), (33, 513), (41, 1001), (9, 777)]:
        img = _img("iid", h * 131 + w, h, w, dt)
        assert np.array_equal(run(gctx, img, n, C4 + OPPOSITE[:2]), oracle.glcm(img, n, C4 + OPPOSITE[:2])), (h, w)
    base = _img("smooth", 97, 120, 1200, dt)
    t = torch.from_numpy(base).cuda()
    for x0, x1 in [(1, 600), (3, 1197), (7, 520)]:
        c = gctx.compute(t[:, x0:x1], n, C4)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(c), oracle.glcm(np.ascontiguousarray(base[:, x0:x1]), n, C4)), (x0, x1)


def offsets_at(d):
    return [(d, 0), (d, -d), (0, -d), (-d, -d)]


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 256])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_distances_up_to_four(gctx, d, n, dt):
    """Offsets at chessboard distance 2..4 take the column walk too (the row
    D above from a ring in shared memory, partner words shifted D pixels):
    all four angles, their opposites, beside distance 1 and distance 5 (the
    general kernel) in one call, on noise and smooth halves."""
    img = _img("smooth", 200 + 10 * d + n, 230, 1037, dt)
    img[:, 600:] = _img("iid", 300 + d + n, 230, 437, dt)
    for offs in (offsets_at(d), [(-dx, -dy) for dx, dy in offsets_at(d)],
                 offsets_at(d) + offsets_at(1) + [(5, 0), (0, -5)]):
        assert np.array_equal(run(gctx, img, n, offs), oracle.glcm(img, n, offs)), (d, offs)


@pytest.mark.parametrize("n", [8, 16, 256])
@pytest.mark.parametrize("h,w", [(1, 1), (2, 3), (3, 2), (4, 4), (5, 5), (7, 513), (70, 17), (33, 1030)])
def test_distances_on_small_and_narrow_images(gctx, h, w, n):
    """Images no larger than the distance, widths around the strips and the
    N = 16 / 256 edge masks (anchors with no partner D to the left or right)."""
    for dt in (np.uint8, np.uint16):
        img = _img("iid", h * 1009 + w + n, h, w, dt)
        offs = offsets_at(2) + offsets_at(4) + [(-3, 0), (0, 3), (3, 3)]
        assert np.array_equal(run(gctx, img, n, offs), oracle.glcm(img, n, offs)), (dt, h, w)


def test_distances_pitched_views_stripes_and_batches(gctx):
    base = _img("smooth", 77, 400, 2100, np.uint8)
    t = torch.from_numpy(base).cuda()
    offs = S.MULTISPECTRAL_OFFSETS
    for x0, x1 in [(0, 1000), (16, 1530), (3, 700)]:
        c = gctx.compute(t[:, x0:x1], 32, offs)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(c), oracle.glcm(np.ascontiguousarray(base[:, x0:x1]), 32, offs)), (x0, x1)
    big = _img("smooth", 78, 3000, 1500, np.uint8)
    big[1500:] = _img("iid", 79, 1500, 1500, np.uint8)
    for n in (8, 32, 256):  # host image in row stripes: the D rows above a stripe come from earlier copies
        c = gctx.compute(big, n, offsets_at(4) + offsets_at(2))
        assert np.array_equal(to_u32(c), oracle.glcm(big, n, offsets_at(4) + offsets_at(2))), n
    u16 = [_img(k, 80 + i, 300, 520, np.uint16) for i, k in enumerate(("iid", "smooth", "constant"))]
    jobs = [dict(image=dev(im), levels=32, offsets=offs, flags=G.GLCM_SYMMETRIC, normalized=True, features=True)
            for im in u16]
    outs = gctx.batch(jobs)
    torch.cuda.synchronize()
    for im, (c, _, _) in zip(u16, outs):
        assert np.array_equal(to_u32(c), oracle.glcm(im, 32, offs))


def test_distance_four_constant_image_all_in_one_bin():
    with G.Context(0, hbm_budget_bytes=1 << 30) as ctx:
        img = np.full((2048, 2048), 200, np.uint8)
        for n in (8, 32, 256):
            offs = offsets_at(4) + offsets_at(3)
            assert np.array_equal(run(ctx, img, n, offs), oracle.glcm(img, n, offs)), n
