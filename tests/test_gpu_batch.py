"""Batched launches: many images of uneven sizes and types in one persistent
launch give, per image, exactly what the image gives alone; the graph
replay gives the same again; the full contention sweep at 4096^2 (the
benchmark's launch) matches the oracle."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32
from featcheck import assert_features, assert_normalized

pytestmark = pytest.mark.gpu


def _jobs(seed=0):
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(9):
        h, w = int(rng.integers(1, 700)), int(rng.integers(1, 1500))
        u16 = k % 3 == 2
        n = int(rng.choice([8, 16, 32, 64, 256]))
        kind = ["iid", "smooth", "constant"][k % 3]
        img = S.image(kind, 100 + k, h, w, np.uint16 if u16 else np.uint8, sigma=3.0)
        offs = S.offsets_for((1, 2)) if k % 2 else S.CONTENTION_OFFSETS
        jobs.append((img, n, offs, G.GLCM_SYMMETRIC if k % 2 else 0))
    return jobs


def test_batch_equals_alone_and_oracle(gctx):
    jobs = _jobs()
    spec = [dict(image=torch.from_numpy(im).cuda(), levels=n, offsets=o, flags=f, normalized=True, features=True)
            for im, n, o, f in jobs]
    for rep in range(3):  # first call captures, later calls replay the graph
        outs = gctx.batch(spec)
        torch.cuda.synchronize()
        for (im, n, o, f), (c, nm, ft) in zip(jobs, outs):
            P = oracle.glcm(im, n, o)
            assert np.array_equal(to_u32(c), P), (im.shape, n, rep)
            alone = gctx.compute(torch.from_numpy(im).cuda(), n, o, f)
            fa = gctx.features(alone, n, symmetric=bool(f & 1))
            torch.cuda.synchronize()
            assert np.array_equal(to_u32(alone), P)
            assert np.array_equal(ft.cpu().numpy(), fa.cpu().numpy())
            sym = bool(f & 1)
            Sm = oracle.symmetrize(P) if sym else P.astype(np.uint64)
            assert_normalized(nm.cpu().numpy(), oracle.normalize(Sm))
            assert_features(ft.cpu().numpy(), oracle.haralick_batch(P, sym), n)


@pytest.mark.slow
def test_contention_sweep_full_size(gctx):
    """The benchmark's batch: 12 images of 4096^2, 4 offsets each, symmetric
    normalized GLCMs and features, one graph launch."""
    jobs = S.contention_jobs(4096)
    spec = [dict(image=torch.from_numpy(j["image"]).cuda(), levels=j["levels"], offsets=j["offsets"],
                 flags=G.GLCM_SYMMETRIC, normalized=True, features=True) for j in jobs]
    gctx.batch(spec)
    outs = gctx.batch(spec)  # graph replay
    torch.cuda.synchronize()
    for j, (c, nm, ft) in zip(jobs, outs):
        P = oracle.glcm(j["image"], j["levels"], j["offsets"])
        assert np.array_equal(to_u32(c), P), (j["kind"], j["levels"])
        assert_features(ft.cpu().numpy(), oracle.haralick_batch(P, True), j["levels"],
                        what=f'{j["kind"]} N={j["levels"]}')
        assert_normalized(nm.cpu().numpy(), oracle.normalize(oracle.symmetrize(P)))


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_batch(gctx, pinned):
    """A batch from host memory (images and results), mixed with one device
    image: staged in groups on the copy stream; every result equals the
    oracle and the same batch from device memory."""
    jobs = _jobs(7)
    spec_h, spec_d = [], []
    for k, (im, n, o, f) in enumerate(jobs):
        t = torch.from_numpy(np.ascontiguousarray(im))
        if pinned:
            t = t.pin_memory()
        img = t.cuda() if k == 3 else t   # one device image in the mix
        outs = [torch.empty((len(o), n, n), dtype=torch.int32), torch.empty((len(o), n, n), dtype=torch.float32),
                torch.empty((len(o), 14), dtype=torch.float32)]
        if pinned:
            outs = [x.pin_memory() for x in outs]
        spec_h.append(dict(image=img, levels=n, offsets=o, flags=f, counts=outs[0], normalized=outs[1],
                           features=outs[2]))
        spec_d.append(dict(image=torch.from_numpy(im).cuda(), levels=n, offsets=o, flags=f, normalized=True,
                           features=True))
    for rep in range(2):
        gctx.batch(spec_h)
        dev = gctx.batch(spec_d)
        torch.cuda.synchronize()
        for (im, n, o, f), h, (c, nm, ft) in zip(jobs, spec_h, dev):
            P = oracle.glcm(im, n, o)
            assert np.array_equal(h["counts"].numpy().view(np.uint32), P), (im.shape, n, rep)
            assert np.array_equal(h["features"].numpy(), ft.cpu().numpy())
            assert np.array_equal(h["normalized"].numpy(), nm.cpu().numpy())


def test_prepared_batch_repeats(gctx):
    """prepare() builds a batch's descriptors once; run() repeats it on the same
    buffers: pinned host images and results in one batch, device ones in
    another, each run equal to the oracle and to batch()."""
    jobs = _jobs(6)
    spec_h, spec_d = [], []
    for im, n, o, f in jobs:
        outs = [torch.empty((len(o), n, n), dtype=torch.int32).pin_memory(),
                torch.empty((len(o), n, n), dtype=torch.float32).pin_memory(),
                torch.empty((len(o), 14), dtype=torch.float32).pin_memory()]
        spec_h.append(dict(image=torch.from_numpy(np.ascontiguousarray(im)).pin_memory(), levels=n, offsets=o,
                           flags=f, counts=outs[0], normalized=outs[1], features=outs[2]))
        spec_d.append(dict(image=torch.from_numpy(im).cuda(), levels=n, offsets=o, flags=f, normalized=True,
                           features=True))
    ph, pd = gctx.prepare(spec_h), gctx.prepare(spec_d)
    want = gctx.batch([dict(s, normalized=True, features=True, counts=None) for s in spec_d])
    torch.cuda.synchronize()
    for rep in range(3):
        gctx.run(ph)
        dev = gctx.run(pd)
        torch.cuda.synchronize()
        for (im, n, o, f), h, (c, nm, ft), (wc, wn, wf) in zip(jobs, spec_h, dev, want):
            P = oracle.glcm(im, n, o)
            assert np.array_equal(h["counts"].numpy().view(np.uint32), P), (im.shape, n, rep)
            assert np.array_equal(to_u32(c), P)
            assert np.array_equal(h["features"].numpy(), wf.cpu().numpy())
            assert np.array_equal(ft.cpu().numpy(), wf.cpu().numpy())
            assert np.array_equal(h["normalized"].numpy(), wn.cpu().numpy())


def test_light_classes_side_by_side(gctx):
    """A batch of N <= 32 uint8 images only: its column-walk classes vote side
    by side, one stream per N (an N with rows at 16-byte starts and at odd
    starts has two classes on one stream), and each N's epilogue follows its
    own votes; some images ask for counts only.  Every result equals the
    oracle and the image alone, on the direct run and on graph replays."""
    rng = np.random.default_rng(77)
    jobs = []
    for k in range(12):
        n = (8, 16, 32)[k % 3]
        h = int(rng.integers(40, 400))
        w = 512 if k % 2 == 0 else int(rng.integers(33, 900)) | 1  # aligned rows, odd widths
        img = S.image(["iid", "smooth", "constant"][k % 3], 300 + k, h, w, np.uint8, sigma=3.0)
        feats = k % 4 != 3
        jobs.append((img, n, feats))
    spec = [dict(image=torch.from_numpy(im).cuda(), levels=n, offsets=S.CONTENTION_OFFSETS,
                 flags=G.GLCM_SYMMETRIC, normalized=f, features=f) for im, n, f in jobs]
    for rep in range(3):
        outs = gctx.batch(spec)
        torch.cuda.synchronize()
        for (im, n, f), (c, nm, ft) in zip(jobs, outs):
            P = oracle.glcm(im, n, S.CONTENTION_OFFSETS)
            assert np.array_equal(to_u32(c), P), (im.shape, n, rep)
            if not f:
                continue
            alone = gctx.compute(torch.from_numpy(im).cuda(), n, S.CONTENTION_OFFSETS, G.GLCM_SYMMETRIC)
            fa = gctx.features(alone, n, symmetric=True)
            torch.cuda.synchronize()
            assert np.array_equal(ft.cpu().numpy(), fa.cpu().numpy()), (im.shape, n, rep)
            assert_normalized(nm.cpu().numpy(), oracle.normalize(oracle.symmetrize(P)))
            assert_features(ft.cpu().numpy(), oracle.haralick_batch(P, True), n, what=f"{im.shape} N={n}")
