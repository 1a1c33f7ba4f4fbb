"""The C ABI library builds, loads on a machine without a GPU, and exports
every function include/glcm.h declares; host-only entry points behave."""
import ctypes

import pytest

import paper_1710_06189_gb300 as G
from paper_1710_06189_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load(build_if_missing=False)


def test_every_declared_symbol_is_exported(lib):
    names = binding.declared_functions()
    assert len(names) >= 10
    raw = ctypes.CDLL(build.LIB)
    for n in names:
        assert hasattr(raw, n), n


def test_binding_covers_the_header(lib):
    assert set(binding.declared_functions()) <= set(binding._PROTOS)


def test_offset_from_angle_matches_eq2_directions(lib):
    # Eq. 2: 0 deg -> right neighbour; 45/90/135 deg -> the row above, to the
    # right / same column / to the left (rows grow downwards).
    assert G.glcm_offset_from_angle(1, 0) == (1, 0)
    assert G.glcm_offset_from_angle(1, 45) == (1, -1)
    assert G.glcm_offset_from_angle(3, 90) == (0, -3)
    assert G.glcm_offset_from_angle(4, 135) == (-4, -4)
    for bad in [(0, 0), (1, 30), (-1, 90)]:
        with pytest.raises(G.GlcmError):
            G.glcm_offset_from_angle(*bad)


def test_status_codes_match_header(lib):
    text = open(binding.HEADER).read()
    for name in ["GLCM_ERR_ARG = -1", "GLCM_ERR_RANGE = -2", "GLCM_ERR_NOMEM = -3", "GLCM_ERR_UNSUPPORTED = -4",
                 "GLCM_ERR_CUDA = -5", "GLCM_ERR_TIMEOUT = -6", "GLCM_ERR_BUSY = -7"]:
        assert name in text
    assert binding.GLCM_ERR_BUSY == -7 and binding.GLCM_SYMMETRIC == 1 and binding.GLCM_INPUT_LEVELS == 4


def test_null_context_arguments_fail_cleanly(lib):
    assert lib.glcm_destroy(None) == 0
    assert lib.glcm_synchronize(None) == binding.GLCM_ERR_ARG
    assert lib.glcm_compute(None, None, 1, 1, 1, 0, 8, None, 0, 0, None, None) == binding.GLCM_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.glcm_create(None, 0, 0, None) == binding.GLCM_ERR_ARG
    assert b"NULL" in lib.glcm_last_error(None)
    del out


def test_create_without_gpu_reports_no_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(G.GlcmError) as ei:
        G.glcm_create(0)
    assert ei.value.status == binding.GLCM_ERR_ARG
