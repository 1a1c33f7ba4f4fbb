"""GLCM counts for N > 256 (up to 4096; N = 1024 quantizes full-range
uint16 by 64 values per level), voted into global counts with warp
aggregation: bit-exact against the oracle (which takes any N) on noise and
smooth uint16 images, uint8 images, levels mode with an out-of-range pixel,
flat-wrap pairs, a batch mixed with N <= 256 images, and the limits (features
and normalized GLCMs need N <= 256; N > 4096 is refused)."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32

pytestmark = pytest.mark.gpu

C4 = S.CONTENTION_OFFSETS


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [257, 512, 1024, 4096])
@pytest.mark.parametrize("kind", ["iid", "smooth"])
def test_wide_levels_u16(gctx, n, kind):
    img = S.image(kind, 700 + n, 300, 517, np.uint16, sigma=6.0)
    offs = C4 + [(-1, 0), (3, -2)]
    c = gctx.compute(dev(img), n, offs)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(c), oracle.glcm(img, n, offs))


def test_wide_levels_u8_levels_mode_flat_and_batch(gctx):
    img = S.iid(71, 200, 333, np.uint8)
    c = gctx.compute(dev(img), 1000, C4)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(c), oracle.glcm(img, 1000, C4))
    lv = (S.iid(72, 90, 130, np.uint16) % 600).astype(np.uint16)
    lv[10, 20] = 700
    out = torch.empty((4, 600, 600), dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError) as e:
        gctx.compute(dev(lv), 600, C4, G.GLCM_INPUT_LEVELS, out=out)
    assert e.value.status == G.GLCM_ERR_RANGE
    assert np.array_equal(to_u32(out), oracle.glcm(lv, 600, C4, levels_mode=True))
    c = gctx.compute(dev(img), 512, C4 + [(5, 0)], G.GLCM_FLAT_WRAP)
    torch.cuda.synchronize()
    assert np.array_equal(to_u32(c), oracle.glcm_flat(img, 512, C4 + [(5, 0)]))
    u16 = S.image("smooth", 73, 256, 700, np.uint16, sigma=3.0)
    jobs = [dict(image=dev(u16), levels=1024, offsets=C4, flags=0),
            dict(image=dev(img), levels=16, offsets=C4, flags=G.GLCM_SYMMETRIC, features=True),
            dict(image=dev(u16), levels=300, offsets=[(1, 0)], flags=0)]
    prepared = gctx.prepare(jobs)
    for rep in range(2):
        res = gctx.run(prepared)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(res[0][0]), oracle.glcm(u16, 1024, C4)), rep
        assert np.array_equal(to_u32(res[1][0]), oracle.glcm(img, 16, C4)), rep
        assert np.array_equal(to_u32(res[2][0]), oracle.glcm(u16, 300, [(1, 0)])), rep


def test_wide_levels_limits(gctx):
    img = dev(S.iid(74, 40, 50, np.uint16))
    with pytest.raises(G.GlcmError) as e:
        gctx.compute(img, 4097, C4)
    assert e.value.status == G.binding.GLCM_ERR_UNSUPPORTED
    with pytest.raises(G.GlcmError) as e:
        gctx.compute(img, 1024, C4, normalized=True)
    assert e.value.status == G.binding.GLCM_ERR_UNSUPPORTED
    with pytest.raises(G.GlcmError) as e:
        gctx.batch([dict(image=img, levels=1024, offsets=C4, features=True)])
    assert e.value.status == G.binding.GLCM_ERR_UNSUPPORTED
