"""glcm_compute_noalloc: the entry point for callers that cannot allocate
device memory while they run (pre-reserved real-time pipelines, code inside a
custom allocator or memory pool, threads that must not block on the
allocator).  Its counts must equal the oracle's and glcm_compute's, bit for
bit, on two calls in a row: the static scratch it reuses keeps the previous
call's contents, so the second call checks that everything that must start
at zero is cleared.  A levels-mode call with an out-of-range pixel must
report GLCM_ERR_RANGE and the clean call after it GLCM_OK (the error word is
cleared per call).  A tall image that wants more scheduling chunks than the
static table holds must still come out exact (the chunks are made coarser).
Runs alone in a fresh process or after the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    ("iid", np.uint8, 777, 1031, 32, [(1, 0), (1, -1), (0, -1), (-1, -1)], 0),
    ("smooth", np.uint16, 300, 513, 256, [(1, 0), (0, -2), (-3, 1)], 0),
    ("iid", np.uint8, 65, 200, 8, [(1, 0), (2, -2), (7, 0), (0, 20)], 0),
    ("constant", np.uint8, 1200, 1100, 256, [(1, 0), (1, -1), (0, -1), (-1, -1)], 0),
    ("iid", np.uint8, 900, 1300, 256, [(1, 0), (1, -1), (0, -1), (-1, -1)], 0),
]


def _image(kind, dtype, h, w, seed):
    import glcm_synth as S
    return S.image(kind, seed, h, w, dtype, sigma=3.0)


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_06189_gb300 import build
    build.build()
    import paper_1710_06189_gb300 as G
    from paper_1710_06189_gb300 import binding
    torch.cuda.init()
    return torch, G, binding


def _noalloc(torch, G, binding, d, n, offs, flags):
    h, w = d.shape
    pitch = d.stride(0) * d.element_size()
    dt = G.GLCM_U8 if d.dtype == torch.uint8 else G.GLCM_U16
    out = torch.full((len(offs), n, n), -1, dtype=torch.int32, device="cuda")
    binding.glcm_compute_noalloc(d, w, h, pitch, dt, n, offs, flags, out)
    return out.cpu().numpy().view(np.uint32)


def test_noalloc_matches_oracle_and_glcm_compute_twice(oracle_lib):
    torch, G, binding = _setup()
    with G.Context(0) as ctx:
        for case_no, (kind, dtype, h, w, n, offs, flags) in enumerate(CASES):
            img = _image(kind, dtype, h, w, 40 + case_no)
            d = torch.from_numpy(img).cuda()
            oracle_counts = oracle_lib.glcm(img, n, offs)
            want = ctx.compute(d, n, offs, flags)
            torch.cuda.synchronize()
            want = want.cpu().numpy().view(np.uint32)
            assert np.array_equal(want, oracle_counts), (kind, n)
            for rep in range(2):
                got = _noalloc(torch, G, binding, d, n, offs, flags)
                assert np.array_equal(got, oracle_counts), (kind, n, rep)


def test_noalloc_levels_mode_range_error_then_clean_call(oracle_lib):
    torch, G, binding = _setup()
    n, offs = 8, [(1, 0), (0, -1)]
    img = np.random.default_rng(77).integers(0, n, size=(130, 260), dtype=np.uint8)
    bad = img.copy()
    bad[64, 100] = n  # one out-of-range pixel: its pairs are skipped
    d_bad = torch.from_numpy(bad).cuda()
    with pytest.raises(G.GlcmError) as ei:
        _noalloc(torch, G, binding, d_bad, n, offs, G.GLCM_INPUT_LEVELS)
    assert ei.value.status == binding.GLCM_ERR_RANGE
    # The counts of the failed call still skip exactly the bad pixel's pairs.
    out = torch.full((len(offs), n, n), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError):
        binding.glcm_compute_noalloc(d_bad, 260, 130, 260, G.GLCM_U8, n, offs, G.GLCM_INPUT_LEVELS, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle_lib.glcm(bad, n, offs, levels_mode=True))
    # The next clean call must not see the previous call's error bit.
    for rep in range(2):
        got = _noalloc(torch, G, binding, torch.from_numpy(img).cuda(), n, offs, G.GLCM_INPUT_LEVELS)
        assert np.array_equal(got, oracle_lib.glcm(img, n, offs, levels_mode=True)), rep


def test_noalloc_coarser_chunks_for_a_tall_image(oracle_lib):
    """512 x 280,000 uint8, N = 2, one offset: one column strip of 8,750 items
    of 32 rows, each its own chunk at first -- more than the 8,192 the static
    chunk table holds, so the call must merge chunks (and still count every
    item exactly once)."""
    torch, G, binding = _setup()
    h, w, n, offs = 280_000, 512, 2, [(1, 0)]
    img = np.random.default_rng(91).integers(0, 256, size=(h, w), dtype=np.uint8)
    d = torch.from_numpy(img).cuda()
    want = oracle_lib.glcm(img, n, offs)
    assert int(want.sum()) == (w - 1) * h
    for rep in range(2):
        got = _noalloc(torch, G, binding, d, n, offs, 0)
        assert np.array_equal(got, want), rep


def test_noalloc_rejects_host_pointers_and_bad_sizes():
    torch, G, binding = _setup()
    img = np.zeros((8, 8), dtype=np.uint8)
    out = torch.empty((1, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError) as ei:
        binding.glcm_compute_noalloc(img, 8, 8, 8, G.GLCM_U8, 8, [(1, 0)], 0, out)
    assert ei.value.status == binding.GLCM_ERR_ARG
    d = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(G.GlcmError) as ei:
        binding.glcm_compute_noalloc(d, 8, 8, 8, G.GLCM_U8, 300, [(1, 0)], 0, out)
    assert ei.value.status == binding.GLCM_ERR_UNSUPPORTED
    with pytest.raises(G.GlcmError) as ei:
        binding.glcm_compute_noalloc(d, 8, 8, 8, G.GLCM_U8, 1, [(1, 0)], 0, out)
    assert ei.value.status == binding.GLCM_ERR_ARG
    with pytest.raises(G.GlcmError) as ei:
        binding.glcm_compute_noalloc(d, 8, 8, 4, G.GLCM_U8, 8, [(1, 0)], 0, out)
    assert ei.value.status == binding.GLCM_ERR_ARG
