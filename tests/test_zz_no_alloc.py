"""glcm_compute_noalloc: the entry point for callers that cannot allocate
device memory while they run (pre-reserved real-time pipelines, code inside a
custom allocator).  Its counts must equal glcm_compute's, bit for bit, on
two calls in a row (the static scratch it reuses keeps the previous call's
contents, so the second call checks that everything that must start at
zero is cleared).  Runs alone in a fresh process or after the other tests."""
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


def test_noalloc_matches_glcm_compute_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_06189_gb300 import build
    build.build()
    import paper_1710_06189_gb300 as G
    from paper_1710_06189_gb300 import binding

    torch.cuda.init()
    with G.Context(0) as ctx:
        for case_no, (kind, dtype, h, w, n, offs, flags) in enumerate(CASES):
            img = _image(kind, dtype, h, w, 40 + case_no)
            d = torch.from_numpy(img).cuda()
            pitch = d.stride(0) * d.element_size()
            dt = G.GLCM_U8 if dtype == np.uint8 else G.GLCM_U16
            want = ctx.compute(d, n, offs, flags)
            torch.cuda.synchronize()
            want = want.cpu().numpy().view(np.uint32)
            for rep in range(2):
                out = torch.full((len(offs), n, n), -1, dtype=torch.int32, device="cuda")
                binding.glcm_compute_noalloc(d, w, h, pitch, dt, n, offs, flags, out)
                got = out.cpu().numpy().view(np.uint32)
                assert np.array_equal(got, want), (kind, n, rep)


def test_noalloc_rejects_host_pointers_and_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_06189_gb300 as G
    from paper_1710_06189_gb300 import binding

    img = np.zeros((8, 8), dtype=np.uint8)
    out = torch.empty((1, 8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(G.GlcmError) as ei:
        binding.glcm_compute_noalloc(img, 8, 8, 8, G.GLCM_U8, 8, [(1, 0)], 0, out)
    assert ei.value.status == binding.GLCM_ERR_ARG
    d = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(G.GlcmError) as ei:
        binding.glcm_compute_noalloc(d, 8, 8, 8, G.GLCM_U8, 300, [(1, 0)], 0, out)
    assert ei.value.status == binding.GLCM_ERR_ARG
