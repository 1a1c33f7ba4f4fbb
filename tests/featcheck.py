"""Tolerance helpers shared by the GPU parity tests.

Features: per feature k, |gpu - oracle| / max(|oracle|, s_k) <= 1e-5.  The
scale floor s_k only matters when the oracle value is below it:
  * s_k = 1 for correlation (f3) and the three correlation measures
    f12-f14, which hover around 0 on independent (iid) GLCMs, where a
    relative error of a value near 0 says nothing;
  * s_k = 1 / N^2 for every other feature.  1 / N^2 is the probability
    resolution of an N x N table (the angular second moment's smallest
    value, and below the inverse difference moment's smallest value
    1 / (1 + (N - 1)^2) only by a factor of about 1); contrast, the sums and
    variances of levels, and the entropies fall below it only for GLCMs with
    almost all mass in one cell, which are then checked to 1e-5 / N^2
    absolute (an exact 0 must come out as 0).
Normalized GLCMs: float32 division of exact integers, so the relative error
is at most 1.5 ulp (3 roundings of half an ulp)."""
import numpy as np

FEATURE_TOL = 1e-5
NORM_RTOL = 4e-7


# Features (0-based) whose floor stays 1: correlation, IMC1, IMC2, MCC.
UNIT_FLOOR = (2, 11, 12, 13)


def feature_scale(levels: int) -> np.ndarray:
    s = np.full(14, 1.0 / (levels * levels))
    s[list(UNIT_FLOOR)] = 1.0
    return s


def map_scale(levels: int) -> np.ndarray:
    """Floors of the four window maps (contrast, ASM, IDM, entropy): 1 / N^2
    each, as for the same features above."""
    return np.full(4, 1.0 / (levels * levels))


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
