"""CUDA path vs the CPU oracle: counts bit-exact, epilogue within tolerance.

Sizes span several column strips, several row bands and ragged tails; the
edge cases are 1x1 images, offsets longer than the image (empty GLCMs),
unaligned pitches, odd widths, non-power-of-two N, wide offsets that take the
per-pixel path, and out-of-range pixels in levels mode."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32
from featcheck import assert_features, assert_normalized

pytestmark = pytest.mark.gpu

C4 = S.CONTENTION_OFFSETS


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(gctx, img, n, offs, flags=0):
    c = gctx.compute(dev(img), n, offs, flags)
    torch.cuda.synchronize()
    return to_u32(c)


def test_plain_512_levels(gctx):
    img, n, offs = S.plain_512()
    got = run(gctx, img, n, offs, G.GLCM_INPUT_LEVELS)
    want = oracle.glcm(img, n, offs, levels_mode=True)
    assert np.array_equal(got, want)
    assert int(got.sum()) == 511 * 512


@pytest.mark.parametrize("kind", ["iid", "smooth", "constant"])
@pytest.mark.parametrize("n", [8, 16, 32, 256])
def test_contention_reduced(gctx, kind, n):
    img = S.image(kind, 11 + n, 777, 1031, np.uint8, sigma=8.0)
    got = run(gctx, img, n, C4)
    assert np.array_equal(got, oracle.glcm(img, n, C4))


@pytest.mark.parametrize("n", [8, 32])
def test_u16_twelve_offsets(gctx, n):
    img = S.iid(5, 333, 1111, np.uint16)
    img[:, 600:] = S.smooth(6, 333, 511, 4.0, np.uint16)
    offs = S.MULTISPECTRAL_OFFSETS
    got = run(gctx, img, n, offs)
    assert np.array_equal(got, oracle.glcm(img, n, offs))


@pytest.mark.parametrize("h,w", [(1, 1), (1, 7), (5, 1), (3, 17), (40, 33), (65, 513), (130, 1000)])
def test_small_and_ragged(gctx, h, w):
    img = S.iid(h * 1000 + w, h, w, np.uint8)
    offs = C4 + [(2, 0), (0, 3), (-4, 4), (4, -4)]
    got = run(gctx, img, 16, offs)
    assert np.array_equal(got, oracle.glcm(img, 16, offs))


def test_unaligned_pitch_and_view(gctx):
    base = S.iid(3, 70, 600, np.uint8)
    view = torch.from_numpy(base).cuda()[:, 3:516]  # pitch 600, odd start: unaligned
    c = gctx.compute(view, 32, C4)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(c), oracle.glcm(np.ascontiguousarray(base[:, 3:516]), 32, C4))


@pytest.mark.parametrize("n", [2, 3, 10, 100, 255])
def test_non_power_of_two_levels(gctx, n):
    img = S.smooth(n, 200, 700, 3.0, np.uint8)
    for dt in (np.uint8, np.uint16):
        im = img.astype(dt) * (257 if dt == np.uint16 else 1)
        got = run(gctx, im, n, C4)
        assert np.array_equal(got, oracle.glcm(im, n, C4)), dt


def test_wide_offsets_and_positive_dy(gctx):
    img = S.iid(9, 300, 900, np.uint8)
    offs = [(7, 0), (-9, 2), (0, 12), (5, 5), (-30, -1), (600, 0), (0, 299), (1000, 0)]
    got = run(gctx, img, 8, offs)
    assert np.array_equal(got, oracle.glcm(img, 8, offs))


def test_levels_mode_range_error_skips_pairs(gctx):
    img = S.iid(4, 64, 640, np.uint8, 0, 8)
    img[10, 100] = 9
    img[33, 5] = 200
    with pytest.raises(G.GlcmError) as ei:
        gctx.compute(dev(img), 8, C4, G.GLCM_INPUT_LEVELS)
    assert ei.value.status == G.binding.GLCM_ERR_RANGE
    out = torch.empty((4, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError):
        gctx.compute(dev(img), 8, C4, G.GLCM_INPUT_LEVELS, out=out)
    want = oracle.glcm(img, 8, C4, levels_mode=True)
    assert np.array_equal(to_u32(out), want)
    # The context stays usable.
    ok = S.iid(4, 64, 640, np.uint8, 0, 8)
    assert np.array_equal(run(gctx, ok, 8, C4, G.GLCM_INPUT_LEVELS), oracle.glcm(ok, 8, C4, levels_mode=True))


def test_u16_levels_mode(gctx):
    img = S.iid(8, 90, 300, np.uint16, 0, 200)
    got = run(gctx, img, 200, C4, G.GLCM_INPUT_LEVELS)
    assert np.array_equal(got, oracle.glcm(img, 200, C4, levels_mode=True))


def test_host_image_stripes(gctx):
    img = S.smooth(21, 2100, 3000, 6.0, np.uint8)  # > 4 MiB: several stripes
    offs = C4 + [(0, 2), (1, 3)]
    c = torch.empty((len(offs), 32, 32), dtype=torch.int32)
    G.glcm_compute(gctx.ctx, img, 3000, 2100, 3000, G.GLCM_U8, 32, offs, 0, c)
    assert np.array_equal(c.numpy().view(np.uint32), oracle.glcm(img, 32, offs))


@pytest.mark.parametrize("x0,w", [(0, 3000), (3, 2999), (13, 1501), (16, 37)])
def test_host_image_pinned_views(gctx, x0, w):
    """Pinned host images, also views whose rows start at any byte and have
    any length: staged by the copy kernel (aligned 16-byte reads realigned on
    the device), through the stripe pipeline and through a host batch."""
    base = torch.from_numpy(S.smooth(22, 2100, 3100, 6.0, np.uint8)).pin_memory()
    view = base[5:2105 - 5, x0:x0 + w]
    img = view.numpy()
    offs = C4 + [(0, 2), (-3, 1)]
    c = torch.empty((len(offs), 32, 32), dtype=torch.int32)
    G.glcm_compute(gctx.ctx, view, w, view.shape[0], view.stride(0), G.GLCM_U8, 32, offs, 0, c)
    want = oracle.glcm(img, 32, offs)
    assert np.array_equal(c.numpy().view(np.uint32), want)
    outs = gctx.batch([dict(image=view, levels=32, offsets=offs, counts=torch.empty_like(c)),
                       dict(image=view, levels=16, offsets=offs, counts=torch.empty((len(offs), 16, 16),
                                                                                    dtype=torch.int32))])
    assert np.array_equal(outs[0][0].numpy().view(np.uint32), want)
    assert np.array_equal(outs[1][0].numpy().view(np.uint32), oracle.glcm(img, 16, offs))


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("n", [8, 32, 256])
def test_normalize_and_features(gctx, sym, n):
    img = S.image("smooth" if n != 256 else "iid", 30 + n, 400, 900, np.uint8, sigma=5.0)
    flags = G.GLCM_SYMMETRIC if sym else 0
    counts, norm = gctx.compute(dev(img), n, C4, flags, normalized=True)
    feats = gctx.features(counts, n, symmetric=sym)
    torch.cuda.synchronize()
    P = oracle.glcm(img, n, C4)
    assert np.array_equal(to_u32(counts), P)
    Sm = oracle.symmetrize(P) if sym else P.astype(np.uint64)
    assert_normalized(norm.cpu().numpy(), oracle.normalize(Sm), f"n={n} sym={sym}")
    assert_features(feats.cpu().numpy(), oracle.haralick_batch(P, sym), n, what=f"n={n} sym={sym}")


@pytest.mark.parametrize("n", [129, 160, 200, 255, 256])
def test_symmetric_features_large_levels(gctx, n):
    """Symmetric GLCMs with N > 128: one cluster of CTAs per GLCM, A' kept by
    rows across it, symmetric Lanczos."""
    imgs = [S.iid(n, 300, 700, np.uint8), S.smooth(n + 1, 300, 700, 2.0, np.uint8),
            S.smooth(n + 2, 300, 700, 8.0, np.uint8), (S.iid(n + 3, 200, 300, np.uint8) & 0xF0),
            (np.indices((64, 96)).sum(0) % 2 * 255).astype(np.uint8),   # checkerboard: f14 = 1
            S.iid(n + 4, 2, 2, np.uint8), S.constant(50, 60)]
    offs = [(1, 0), (1, -1), (0, -1), (-1, -1), (3, -3)]
    for k, img in enumerate(imgs):
        counts, norm = gctx.compute(dev(img), n, offs, G.GLCM_SYMMETRIC, normalized=True)
        feats = gctx.features(counts, n, symmetric=True)
        torch.cuda.synchronize()
        P = oracle.glcm(img, n, offs)
        assert np.array_equal(to_u32(counts), P)
        assert_normalized(norm.cpu().numpy(), oracle.normalize(oracle.symmetrize(P)), f"n={n} img={k}")
        assert_features(feats.cpu().numpy(), oracle.haralick_batch(P, True), n, what=f"n={n} img={k}")


def test_cluster_epilogue_large_totals_and_mixed_launch(gctx):
    """Symmetric GLCMs with 128 < N <= 256 take one cluster of CTAs each: count
    matrices whose symmetric total passes 2^32 (S entries beyond 32 bits, the
    rounded numerator), sparse and single-cell supports, in one call beside
    jobs of the one-CTA epilogue; every GLCM again alone, bit-identical."""
    rng = np.random.default_rng(4242)
    for n in (129, 200, 256):
        mats = [rng.integers(0, 1 << 24, size=(n, n), dtype=np.uint64).astype(np.uint32),
                (rng.random((n, n)) < 0.02) * rng.integers(1, 1 << 31, size=(n, n)),
                np.zeros((n, n), np.uint64)]
        mats[2][n - 1, 0] = 3_000_000_000
        mats = np.stack([m.astype(np.uint32) for m in mats])
        c = torch.from_numpy(mats.view(np.int32)).cuda()
        f = gctx.features(c, n, symmetric=True)
        torch.cuda.synchronize()
        assert_features(f.cpu().numpy(), oracle.haralick_batch(mats, True), n, what=f"n={n} large totals")
        for k in range(len(mats)):
            alone = gctx.features(c[k:k + 1], n, symmetric=True)
            torch.cuda.synchronize()
            assert np.array_equal(alone.cpu().numpy()[0], f.cpu().numpy()[k]), (n, k)
    # One batch: N = 256 and N = 64 symmetric feature jobs, and N = 256 plain.
    img = S.smooth(77, 300, 600, 3.0, np.uint8)
    jobs = [dict(image=dev(img), levels=256, offsets=C4, flags=G.GLCM_SYMMETRIC, features=True),
            dict(image=dev(img), levels=64, offsets=C4, flags=G.GLCM_SYMMETRIC, features=True),
            dict(image=dev(img), levels=256, offsets=C4[:2], flags=0, features=True)]
    outs = gctx.batch(jobs)
    torch.cuda.synchronize()
    for jb, (c, _, f) in zip(jobs, outs):
        P = oracle.glcm(img, jb["levels"], jb["offsets"])
        assert np.array_equal(to_u32(c), P)
        assert_features(f.cpu().numpy(), oracle.haralick_batch(P, jb["flags"] == G.GLCM_SYMMETRIC), jb["levels"],
                        what=f"batch n={jb['levels']}")


def test_features_of_special_matrices(gctx):
    n = 16
    mats = np.zeros((5, n, n), dtype=np.uint32)
    mats[1, 3, 3] = 1000                        # one-hot
    mats[2] = np.eye(n, dtype=np.uint32) * 7    # diagonal
    mats[3] = 5                                 # uniform
    px = np.arange(1, n + 1)
    mats[4] = np.outer(px, px[::-1])            # independent
    c = torch.from_numpy(mats.view(np.int32)).cuda()
    f = gctx.features(c, n).cpu().numpy()
    want = oracle.haralick_batch(mats, False)
    assert_features(f, want, n, what="special")
    assert np.all(f[0] == 0)


@pytest.mark.parametrize("n", [2, 5, 8, 16, 31, 32])
def test_features_small_supports(gctx, n):
    """Supports of at most 32 levels (f14 by repeated squaring of A'^T A'):
    block-diagonal GLCMs whose top singular values of A' repeat (two and
    three disconnected level groups give one and two extra singular values
    of exactly 1), rectangular supports (anchor and partner level sets
    differ), a total of 1, and random dense counts, plain and symmetric."""
    rng = np.random.default_rng(700 + n)
    mats = []
    for groups in (2, 3):
        m = np.zeros((n, n), dtype=np.uint32)
        edges = np.linspace(0, n, groups + 1).astype(int)
        for a, b in zip(edges[:-1], edges[1:]):
            if b > a:
                m[a:b, a:b] = rng.integers(1, 50, (b - a, b - a))
        mats.append(m)
    rect = np.zeros((n, n), dtype=np.uint32)
    rect[: max(1, n // 2), n // 3:] = rng.integers(0, 9, (max(1, n // 2), n - n // 3))
    mats.append(rect)
    one = np.zeros((n, n), dtype=np.uint32)
    one[n - 1, 0] = 1
    mats.append(one)
    mats.append(rng.integers(0, 1000, (n, n)).astype(np.uint32))
    mats.append(rng.integers(0, 3, (n, n)).astype(np.uint32) * (rng.random((n, n)) < 0.3))
    big = rng.integers(0, 1 << 22, (n, n)).astype(np.uint32)   # total near 2^32 / 4 at n = 32
    mats.append(big)
    mats = np.stack(mats).astype(np.uint32)
    for sym in (False, True):
        if sym and np.any(mats.astype(np.uint64).sum(axis=(1, 2)) * 2 >= (1 << 32)):
            mats = mats.copy()
            mats[-1] //= 4
        c = torch.from_numpy(mats.view(np.int32)).cuda()
        f = gctx.features(c, n, symmetric=sym).cpu().numpy()
        assert_features(f, oracle.haralick_batch(mats, sym), n, what=f"n={n} sym={sym}")


def test_naive_scheme1_matches(gctx):
    img = S.smooth(2, 300, 400, 4.0, np.uint8)
    c = torch.empty((8, 8), dtype=torch.int32, device="cuda")
    d = dev(img)
    for off in C4:
        G.glcm_compute_naive(gctx.ctx, d, 400, 300, 400, G.GLCM_U8, 8, off, 0, c)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(c), oracle.glcm(img, 8, [off])[0])


@pytest.mark.parametrize("n", [8, 16, 32, 64, 256])
def test_every_vote_config_is_exact(gctx, n):
    """All histogram layouts, copy counts, thread counts and level splits
    give the same counts (the autotuner may pick any of them)."""
    img = S.smooth(77, 300, 1100, 2.0, np.uint8)
    img[:, 500:] = S.iid(78, 300, 600, np.uint8)
    offs = C4 + [(2, -2)]
    want = oracle.glcm(img, n, offs)
    d = dev(img)
    tried = 0
    for threads in (1024, 256):
        for r in (5, 3, 0):
            for layout in (0, 1, 2, 3):
                try:
                    G.glcm_set_vote_config(gctx.ctx, n, len(offs), G.GLCM_U8, threads, r, layout, 64)
                except G.GlcmError:
                    continue  # does not fit shared memory
                c = gctx.compute(d, n, offs)
                torch.cuda.synchronize()
                assert np.array_equal(to_u32(c), want), (threads, r, layout)
                tried += 1
    G.glcm_set_vote_config(gctx.ctx, n, len(offs), G.GLCM_U8, 0, 0, 0, 0)
    assert tried >= 3


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("n", [256, 255, 8])
def test_packed_halves_spill(gctx, n, dtype):
    """Packed 16-bit halves (layout 3): images whose votes pile into one or
    two bins, millions of votes each, in the lower and the upper half of the
    packed words, for every thread count.  Any half that wrapped between two
    spills would lose 65536 votes."""
    h, w = 1536, 1400
    top = np.iinfo(dtype).max
    img = np.full((h, w), top // 5, dtype)         # a lower-half level
    img[:, 700:] = top - top // 7                    # an upper-half level
    img[::97, :] = top // 2                          # a few rows elsewhere
    offs = C4 + [(3, 2)]
    want = oracle.glcm(img, n, offs)
    assert want.max() > 4 * 65536
    d = dev(img)
    dt = G.GLCM_U8 if dtype == np.uint8 else G.GLCM_U16
    for threads in (1024, 512, 256):
        G.glcm_set_vote_config(gctx.ctx, n, len(offs), dt, threads, 0, 3, 0)
        c = gctx.compute(d, n, offs)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(c), want), threads
    G.glcm_set_vote_config(gctx.ctx, n, len(offs), dt, 0, 0, 0, 0)
