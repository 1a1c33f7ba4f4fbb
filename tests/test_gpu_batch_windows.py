"""glcm_compute_batch_windows: images and sliding-window jobs in one CUDA-graph
launch (config 4's shape at a reduced size).  The direct first call and two
graph replays must give the oracle's counts for every image and window, and
window maps within the feature tolerance."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32
import featcheck

pytestmark = pytest.mark.gpu

C4 = S.CONTENTION_OFFSETS


def test_images_and_windows_in_one_graph(gctx):
    rng = np.random.default_rng(11)
    imgs, jobs = [], []
    for k in range(12):
        side = int(rng.integers(40, 400))
        n = int(rng.choice([8, 16, 32]))
        im = S.image("iid" if k % 2 else "smooth", 300 + k, side, side + k, np.uint8, 4.0)
        imgs.append((im, n))
        jobs.append(dict(image=torch.from_numpy(im).cuda(), levels=n, offsets=C4, flags=G.GLCM_SYMMETRIC,
                         features=True))
    wimg = S.smooth(321, 140, 190, 4.0, np.uint8)
    wd = torch.from_numpy(wimg).cuda()
    windows = [dict(image=wd, levels=16, win=15, stride=4, offsets=C4, flags=G.GLCM_SYMMETRIC, counts=True,
                    maps=True),
               dict(image=wd, levels=8, win=9, stride=3, offsets=[(1, 0), (0, -1)], flags=0, counts=True,
                    maps=False)]
    pw = gctx.prepare_batch_windows(jobs, windows)
    for rep in range(3):
        outs, wouts = gctx.run_batch_windows(pw)
        torch.cuda.synchronize()
        for (im, n), (c, _, ft) in zip(imgs, outs):
            P = oracle.glcm(im, n, C4)
            assert np.array_equal(to_u32(c), P), rep
            featcheck.assert_features(ft.cpu().numpy(), oracle.haralick_batch(P, True), n)
        for w, (c, m) in zip(windows, wouts):
            want = oracle.window_glcm(wimg, w["levels"], w["offsets"], w["win"], w["stride"])
            got = to_u32(c).reshape(want.shape)
            assert np.array_equal(got, want), (w["win"], rep)
            if m is not None:
                maps = oracle.window_maps(want, symmetric=True)
                nw = want.shape[0]
                g = m.cpu().numpy().reshape(4, len(w["offsets"]), nw).transpose(0, 2, 1).astype(np.float64)
                err = np.abs(g - maps) / np.maximum(np.abs(maps), featcheck.map_scale(16)[:, None, None])
                assert err.max() <= 1e-5, err.max()


def test_windows_only_batch(gctx):
    wimg = S.iid(5, 64, 80, np.uint8)
    pw = gctx.prepare_batch_windows([], [dict(image=torch.from_numpy(wimg).cuda(), levels=4, win=7, stride=2,
                                               offsets=[(1, 0)], counts=True, maps=False)])
    for _ in range(2):
        _, wouts = gctx.run_batch_windows(pw)
        torch.cuda.synchronize()
        want = oracle.window_glcm(wimg, 4, [(1, 0)], 7, 2)
        assert np.array_equal(to_u32(wouts[0][0]).reshape(want.shape), want)
