"""Tolerance helpers shared by the GPU parity tests.

Features: per feature k, |gpu - oracle| / max(|oracle|, s_k) <= 1e-5, with
the scale floor s_k = 1/N^2 for the angular second moment (its smallest
possible value) and 1 for every other feature (levels, log-units and
correlations are all O(1) quantities; a zero oracle value is then checked
absolutely).  Normalized GLCMs: float32 division of exact integers, so the
relative error is at most 1.5 ulp (3 roundings of half an ulp)."""
import numpy as np

FEATURE_TOL = 1e-5
NORM_RTOL = 4e-7


def feature_scale(levels: int) -> np.ndarray:
    s = np.ones(14)
    s[0] = 1.0 / (levels * levels)
    return s


def feature_errors(gpu: np.ndarray, want: np.ndarray, levels: int) -> np.ndarray:
    """Scaled error per feature (max over GLCMs), shape (14,)."""
    g = np.asarray(gpu, dtype=np.float64).reshape(-1, 14)
    w = np.asarray(want, dtype=np.float64).reshape(-1, 14)
    err = np.abs(g - w) / np.maximum(np.abs(w), feature_scale(levels)[None, :])
    return err.max(axis=0) if len(err) else np.zeros(14)


def relative_errors(gpu: np.ndarray, want: np.ndarray) -> np.ndarray:
    g = np.asarray(gpu, dtype=np.float64).reshape(-1, 14)
    w = np.asarray(want, dtype=np.float64).reshape(-1, 14)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(w != 0, np.abs(g - w) / np.abs(w), np.abs(g - w))
    return r.max(axis=0) if len(r) else np.zeros(14)


def assert_features(gpu, want, levels, tol=FEATURE_TOL, what=""):
    e = feature_errors(gpu, want, levels)
    bad = np.nonzero(e > tol)[0]
    assert len(bad) == 0, f"{what} features {[(int(k) + 1, float(e[k])) for k in bad]} exceed {tol}"
    return e


def assert_normalized(gpu, want, what=""):
    g = np.asarray(gpu, dtype=np.float64)
    w = np.asarray(want, dtype=np.float64)
    ok = np.abs(g - w) <= NORM_RTOL * np.abs(w)
    assert ok.all(), f"{what} normalized differs at {np.argwhere(~ok)[:5].tolist()}"
