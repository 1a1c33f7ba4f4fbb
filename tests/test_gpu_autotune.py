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


def test_tune_batch_on_the_batch_itself(tmp_path):
    """tune_batch times whole runs of a mixed batch per class and candidate;
    every class gets a config (the planner's default when nothing beats it by
    the margin), and the batch stays bit-exact under the chosen configs."""
    C4 = S.CONTENTION_OFFSETS
    specs = [("iid", 8), ("smooth", 16), ("iid", 256), ("smooth", 256)]
    imgs = [S.image(k, 40 + n, 256, 640, np.uint8, sigma=8.0) for k, n in specs]
    with G.Context(0, hbm_budget_bytes=2 << 30) as ctx:
        jobs = [dict(image=torch.from_numpy(im).cuda(), levels=n, offsets=C4, flags=G.GLCM_SYMMETRIC,
                     features=True) for im, (_, n) in zip(imgs, specs)]
        cache = autotune.TuneCache(str(tmp_path / "b.json"))
        chosen = autotune.tune_batch(ctx, jobs, reps=2, cache=cache, gpu="test")
        assert set(chosen) == {autotune.class_key(n, 4, G.GLCM_U8) for n in (8, 16, 256)}
        for cfg in chosen.values():
            assert cfg["ms"] > 0 and cfg["ms"] <= cfg["default_ms"] * 1.0001
        outs = ctx.batch(jobs)
        torch.cuda.synchronize()
        for im, (_, n), (c, _, _) in zip(imgs, specs, outs):
            assert np.array_equal(to_u32(c), oracle.glcm(im, n, C4))
