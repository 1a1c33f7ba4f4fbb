"""The autotuner on the GPU: it times feasible configs, applies the fastest,
and the counts under the chosen config stay bit-exact with the oracle."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from paper_1710_06189_gb300 import autotune
from conftest import to_u32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [16, 256])
def test_tune_applies_an_exact_config(gctx, n, tmp_path):
    C4 = S.CONTENTION_OFFSETS
    imgs = [S.image(k, 3 + n, 300, 700, np.uint8, sigma=8.0) for k in ("iid", "smooth")]
    dimgs = [torch.from_numpy(i).cuda() for i in imgs]
    ctx = G.Context(0, hbm_budget_bytes=2 << 30)
    try:
        cache = autotune.TuneCache(str(tmp_path / "t.json"))
        chosen = autotune.tune_classes(ctx, {(n, tuple(C4)): dimgs}, cache=cache, gpu="test", reps=1)
        key = autotune.class_key(n, 4, G.GLCM_U8)
        assert key in chosen and chosen[key]["ms"] > 0
        assert autotune.TuneCache(cache.path).get("test", key) == chosen[key]
        for img, d in zip(imgs, dimgs):
            got = to_u32(ctx.compute(d, n, C4))
            assert np.array_equal(got, oracle.glcm(img, n, C4))
        # A second context takes the config from the cache without timing.
        ctx2 = G.Context(0, hbm_budget_bytes=1 << 30)
        try:
            assert cache.apply(ctx2, "test", n, 4, G.GLCM_U8)
            got = to_u32(ctx2.compute(dimgs[0], n, C4))
            assert np.array_equal(got, oracle.glcm(imgs[0], n, C4))
        finally:
            ctx2.close()
    finally:
        ctx.close()
