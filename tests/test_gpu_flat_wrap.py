"""GLCM_FLAT_WRAP (Eq. 2 on the row-major buffer, pairs across row ends)
against the oracle's flat-wrap counts, bit for bit: both vote kernels (the
column walk for distance-1 offsets, the general kernel for the rest), offsets
wider than the image, uint8 and uint16, pitched device images, host images in
stripes, batches and levels-mode range errors."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32

pytestmark = pytest.mark.gpu

C4 = S.CONTENTION_OFFSETS
F = G.GLCM_FLAT_WRAP


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [8, 16, 256, 10])
@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_flat_wrap_matches_oracle(gctx, n, dt):
    img = S.image("smooth", 60 + n, 157, 301, dt, sigma=4.0)
    img[:, 150:] = S.iid(61 + n, 157, 151, dt)
    offs = C4 + [(-1, 0), (0, 1), (3, 2), (-2, -3), (5, 0), (301 + 2, -1), (-(301 + 5), 1)]
    c = gctx.compute(dev(img), n, offs, F)
    torch.cuda.synchronize()
    got = to_u32(c)
    want = oracle.glcm_flat(img, n, offs)
    for k in range(len(offs)):
        assert np.array_equal(got[k], want[k]), offs[k]
    # Without the flag the same call gives the in-rectangle counts.
    c = gctx.compute(dev(img), n, offs, 0)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(c), oracle.glcm(img, n, offs))


def test_flat_wrap_pitched_view_and_host_stripes(gctx):
    base = S.image("iid", 70, 600, 1024, np.uint8)
    t = torch.from_numpy(base).cuda()[:, 16:1000]  # pitch 1024, width 984
    c = gctx.compute(t, 16, C4 + [(7, -2)], F)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(c), oracle.glcm_flat(np.ascontiguousarray(base[:, 16:1000]), 16, C4 + [(7, -2)]))
    big = S.image("smooth", 71, 2500, 1800, np.uint8, sigma=6.0)  # host image: streamed in row stripes
    for n in (8, 32):
        c = gctx.compute(big, n, C4 + [(1, 1)], F)
        assert np.array_equal(to_u32(c), oracle.glcm_flat(big, n, C4 + [(1, 1)])), n


def test_flat_wrap_in_a_batch_and_levels_range(gctx):
    imgs = [S.image("iid", 80 + k, 100 + 37 * k, 220 + 91 * k, np.uint8) for k in range(4)]
    jobs = [dict(image=dev(im), levels=n, offsets=C4 + [(2, 0)], flags=F | G.GLCM_SYMMETRIC, features=True)
            for im, n in zip(imgs, (8, 16, 32, 256))]
    prepared = gctx.prepare(jobs)
    for rep in range(2):
        res = gctx.run(prepared)
        torch.cuda.synchronize()
        for im, jb, (c, _, _) in zip(imgs, jobs, res):
            assert np.array_equal(to_u32(c), oracle.glcm_flat(im, jb["levels"], jb["offsets"])), rep
    lv = np.random.default_rng(5).integers(0, 8, size=(90, 120)).astype(np.uint8)
    lv[40, 119] = 9  # the last pixel of a row: its flat partners are in the next row
    with pytest.raises(G.GlcmError) as e:
        gctx.compute(dev(lv), 8, C4, F | G.GLCM_INPUT_LEVELS)
    assert e.value.status == G.GLCM_ERR_RANGE
    out = torch.empty((4, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError):
        gctx.compute(dev(lv), 8, C4, F | G.GLCM_INPUT_LEVELS, out=out)
    assert np.array_equal(to_u32(out), oracle.glcm_flat(lv, 8, C4, levels_mode=True))
