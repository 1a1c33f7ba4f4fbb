"""Host logic of the vote-kernel autotuner: class keys and the JSON cache."""
import json

from paper_1710_06189_gb300 import autotune
from paper_1710_06189_gb300 import binding as B


def test_class_key_separates_pixel_types_and_offsets():
    a = autotune.class_key(16, 4, B.GLCM_U8)
    b = autotune.class_key(16, 4, B.GLCM_U16)
    c = autotune.class_key(16, 12, B.GLCM_U8)
    assert len({a, b, c}) == 3


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    cache = autotune.TuneCache(path)
    assert cache.get("gpu", "k") is None
    cache.put("gpu", "k", {"threads": 512, "log2_copies": 5, "layout": 1, "band_rows": 32, "ms": 0.25,
                           "tried": [1, 2]})
    cache.save()
    again = autotune.TuneCache(path)
    assert again.get("gpu", "k") == {"threads": 512, "log2_copies": 5, "layout": 1, "band_rows": 32, "ms": 0.25}
    assert again.get("other", "k") is None
    with open(path) as f:
        assert "tried" not in json.load(f)["gpu"]["k"]


def test_default_candidates_are_valid_shapes():
    for threads, r, layout in autotune.DEFAULT_CANDIDATES:
        assert threads % 32 == 0 and 64 <= threads <= 1024
        assert 0 <= r <= 5 and layout in (0, 1, 2, 3, 4)
    assert autotune.DEFAULT_CANDIDATES[0][2] == 4  # the column-walk kernel is tried first
    for layout, bands in autotune.BAND_CANDIDATES.items():
        assert bands[0] == 0 and all(b > 0 for b in bands[1:])
        if layout != 4:
            assert max(bands) <= 64  # the general kernel's tiles hold 64 anchor rows
