"""The serving loop (glcm_server_*): every request's result in a mixed,
continuously batched stream equals the request alone and the oracle;
admission is bounded by the arena; errors belong to their own request."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from featcheck import assert_features, assert_normalized

pytestmark = pytest.mark.gpu


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _stream(n=14, seed=S.BASE_SEED + 900):
    reqs = S.request_stream(n, 1000.0, lo=48, hi=700, seed=seed)
    return [(S.image(r.kind, r.seed, r.side, r.side + (r.rid % 5), np.uint8, 4.0), r.levels, r.offsets,
             G.GLCM_SYMMETRIC if r.rid % 2 else 0) for r in reqs]


def _u32(t):
    return t.numpy().view(np.uint32)


def test_mix_equals_alone_and_oracle():
    items = _stream()
    with G.Server(0, hbm_budget_bytes=256 << 20, lanes=2) as srv:
        imgs = [_pinned(im) for im, _, _, _ in items]
        mix = [srv.submit(im, n, o, f, normalized=True, features=True) for im, (_, n, o, f) in zip(imgs, items)]
        mixed = []
        for t in mix:
            st, lat, outs = srv.wait(t)
            assert st == G.GLCM_OK, srv.last_error()
            assert lat >= 0
            mixed.append(outs)
        for im, (a, n, o, f), (c, nm, ft) in zip(imgs, items, mixed):
            st, _, (c1, nm1, ft1) = srv.wait(srv.submit(im, n, o, f, normalized=True, features=True))
            assert st == G.GLCM_OK
            P = oracle.glcm(a, n, o)
            assert np.array_equal(_u32(c), P), (a.shape, n, o)
            assert np.array_equal(_u32(c1), P)
            assert np.array_equal(ft.numpy(), ft1.numpy())
            assert np.array_equal(nm.numpy(), nm1.numpy())
            sym = bool(f & G.GLCM_SYMMETRIC)
            Sm = oracle.symmetrize(P) if sym else P.astype(np.uint64)
            assert_normalized(nm.numpy(), oracle.normalize(Sm))
            assert_features(ft.numpy(), oracle.haralick_batch(P, sym), n)
        s = srv.stats()
        assert s["completed"] == 2 * len(items) and s["failed"] == 0
        assert s["batches"] >= 1 and s["kernel_launches"] >= s["batches"]


def test_admission_bounded_by_arena():
    arena = 6 << 20
    with G.Server(0, hbm_budget_bytes=arena, lanes=2) as srv:
        imgs = [S.image("iid" if k % 2 else "smooth", 40 + k, 1024, 1000, np.uint8, 4.0) for k in range(20)]
        offs = S.CONTENTION_OFFSETS
        ts = [srv.submit(_pinned(im), 16, offs) for im in imgs]
        for im, t in zip(imgs, ts):
            st, _, (c, _, _) = srv.wait(t)
            assert st == G.GLCM_OK
            assert np.array_equal(_u32(c), oracle.glcm(im, 16, offs))
        s = srv.stats()
        assert s["arena_peak"] <= s["arena_bytes"] <= arena
        assert s["completed"] == 20
        big = np.zeros((4096, 4096), np.uint8)
        with pytest.raises(G.GlcmError) as e:
            srv.submit(big, 8, offs)
        assert e.value.status == G.GLCM_ERR_NOMEM


def test_range_error_is_the_requests_own():
    good = S.iid(3, 200, 300, np.uint8) % 8
    bad = good.copy()
    bad[17, 33] = 9
    offs = [(1, 0), (0, -1)]
    with G.Server(0, hbm_budget_bytes=64 << 20) as srv:
        ts = [srv.submit(_pinned(im), 8, offs, G.GLCM_INPUT_LEVELS) for im in (good, bad, good)]
        res = [srv.wait(t) for t in ts]
        assert [r[0] for r in res] == [G.GLCM_OK, G.GLCM_ERR_RANGE, G.GLCM_OK]
        for r in (res[0], res[2]):
            assert np.array_equal(_u32(r[2][0]), oracle.glcm(good, 8, offs, levels_mode=True))


def test_pageable_buffers_and_device_pointers():
    im = S.smooth(8, 333, 517, 3.0, np.uint8)
    offs = S.offsets_for((1, 2))
    with G.Server(0, hbm_budget_bytes=64 << 20, lanes=1) as srv:
        st, _, (c, _, ft) = srv.wait(srv.submit(im, 32, offs, G.GLCM_SYMMETRIC, features=True, pin=False))
        assert st == G.GLCM_OK
        P = oracle.glcm(im, 32, offs)
        assert np.array_equal(_u32(c), P)
        assert_features(ft.numpy(), oracle.haralick_batch(P, True), 32)
        with pytest.raises(G.GlcmError) as e:
            srv.submit(torch.from_numpy(im).cuda(), 32, offs)
        assert e.value.status == G.binding.GLCM_ERR_ARG


def test_close_finishes_admitted_work():
    srv = G.Server(0, hbm_budget_bytes=64 << 20)
    ims = [_pinned(S.iid(k, 512, 512, np.uint8)) for k in range(6)]
    for im in ims:
        srv.submit(im, 16, S.CONTENTION_OFFSETS)
    srv.close()  # must return: admitted requests finish, queued ones are dropped
