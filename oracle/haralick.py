"""Float64 oracle for the GLCM epilogue and the 14 Haralick features.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names the fourteen texture statistics that Haralick extracted from
each GLCM (Sec. I, introduction, citing Haralick's 1973 paper) but defines
none of them.  They are written out here from their textbook definitions,
term by term, in float64, with natural logarithms and 0 * ln 0 = 0.  Levels
are 0-based, i, j in {0, ..., N-1}.

Notation: p is the normalized GLCM, p_x(i) = sum_j p(i,j), p_y(j) =
sum_i p(i,j), p_{x+y}(k) = sum over i+j = k (k = 0..2N-2), p_{x-y}(k) = sum
over |i-j| = k (k = 0..N-1); mu_x, mu_y, sigma_x, sigma_y are the mean and
standard deviation of p_x and p_y; HX, HY their entropies; HXY the entropy
of p; HXY1 = -sum p(i,j) ln(p_x(i) p_y(j)); HXY2 = -sum p_x(i) p_y(j)
ln(p_x(i) p_y(j)).

  f1  angular second moment   sum p^2
  f2  contrast                sum (i-j)^2 p
  f3  correlation             (sum i j p - mu_x mu_y) / (sigma_x sigma_y); 1 when the
                              denominator is 0
  f4  sum of squares          sum (i - mu_x)^2 p
  f5  inverse difference mom. sum p / (1 + (i-j)^2)
  f6  sum average             sum k p_{x+y}(k)
  f7  sum variance            sum (k - f6)^2 p_{x+y}(k)
  f8  sum entropy             -sum p_{x+y} ln p_{x+y}
  f9  entropy                 -sum p ln p
  f10 difference variance     variance of p_{x-y}
  f11 difference entropy      -sum p_{x-y} ln p_{x-y}
  f12 info. meas. corr. 1     (HXY - HXY1) / max(HX, HY); 0 when the denominator is 0
  f13 info. meas. corr. 2     sqrt(1 - exp(-2 (HXY2 - HXY))), argument clamped at 0
  f14 max. correlation coef.  sqrt(second largest eigenvalue of
                              Q(i,j) = sum_k p(i,k) p(j,k) / (p_x(i) p_y(k)))
                              over the rows and columns where p_x, p_y > 0; Q's
                              eigenvalues are taken from the symmetric matrix
                              D^-1/2 P D_y^-1 P^T D^-1/2 (same spectrum); 0 when
                              fewer than two eigenvalues exist.

An all-zero GLCM (no pixel pairs) normalizes to zeros and has all features 0.
"""
from __future__ import annotations

import numpy as np

FEATURE_NAMES = (
    "asm", "contrast", "correlation", "sum_of_squares", "idm", "sum_average",
    "sum_variance", "sum_entropy", "entropy", "difference_variance",
    "difference_entropy", "imc1", "imc2", "mcc",
)

# Maps computed for each sliding window (local texture maps).
WINDOW_MAP_NAMES = ("contrast", "asm", "idm", "entropy")


def symmetrize(P: np.ndarray) -> np.ndarray:
    """S = P + P^T (counts stay integers; uint64 to avoid any overflow)."""
    P = np.asarray(P, dtype=np.uint64)
    return P + P.swapaxes(-1, -2)


def normalize(S: np.ndarray) -> np.ndarray:
    """p = S / sum(S) in float64; an all-zero matrix stays zero."""
    S = np.asarray(S, dtype=np.float64)
    tot = S.sum(axis=(-1, -2), keepdims=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        p = np.where(tot > 0, S / np.where(tot > 0, tot, 1.0), 0.0)
    return p


def _plogp(v: np.ndarray) -> np.ndarray:
    out = np.zeros_like(v, dtype=np.float64)
    nz = v > 0
    out[nz] = v[nz] * np.log(v[nz])
    return out


def haralick(p: np.ndarray) -> np.ndarray:
    """The 14 features of one normalized N x N GLCM, float64, in f1..f14 order."""
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    f = np.zeros(14, dtype=np.float64)
    if p.sum() <= 0:
        return f
    i = np.arange(n, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    lv = np.arange(n, dtype=np.float64)
    px = p.sum(axis=1)
    py = p.sum(axis=0)

    ii = np.arange(n)[:, None] + np.zeros((1, n), dtype=np.int64)
    jj = np.zeros((n, 1), dtype=np.int64) + np.arange(n)[None, :]
    p_sum = np.zeros(2 * n - 1)
    np.add.at(p_sum, (ii + jj).reshape(-1), p.reshape(-1))
    p_diff = np.zeros(n)
    np.add.at(p_diff, np.abs(ii - jj).reshape(-1), p.reshape(-1))
    ks = np.arange(2 * n - 1, dtype=np.float64)
    kd = np.arange(n, dtype=np.float64)

    mu_x = float((lv * px).sum())
    mu_y = float((lv * py).sum())
    sd_x = float(np.sqrt(((lv - mu_x) ** 2 * px).sum()))
    sd_y = float(np.sqrt(((lv - mu_y) ** 2 * py).sum()))

    f[0] = (p * p).sum()
    f[1] = ((i - j) ** 2 * p).sum()
    if sd_x * sd_y > 0:
        f[2] = ((i * j * p).sum() - mu_x * mu_y) / (sd_x * sd_y)
    else:
        f[2] = 1.0
    f[3] = ((i - mu_x) ** 2 * p).sum()
    f[4] = (p / (1.0 + (i - j) ** 2)).sum()
    f[5] = (ks * p_sum).sum()
    f[6] = ((ks - f[5]) ** 2 * p_sum).sum()
    f[7] = -_plogp(p_sum).sum()
    hxy = -_plogp(p).sum()
    f[8] = hxy
    mean_d = (kd * p_diff).sum()
    f[9] = ((kd - mean_d) ** 2 * p_diff).sum()
    f[10] = -_plogp(p_diff).sum()

    hx = -_plogp(px).sum()
    hy = -_plogp(py).sum()
    q = px[:, None] * py[None, :]
    nzp = p > 0
    hxy1 = -(p[nzp] * np.log(q[nzp])).sum()
    nzq = q > 0
    hxy2 = -(q[nzq] * np.log(q[nzq])).sum()
    den = max(hx, hy)
    f[11] = (hxy - hxy1) / den if den > 0 else 0.0
    f[12] = np.sqrt(max(0.0, 1.0 - np.exp(-2.0 * (hxy2 - hxy))))

    rows = px > 0
    cols = py > 0
    if rows.sum() >= 2:
        ps = p[np.ix_(rows, cols)]
        dx_ = 1.0 / np.sqrt(px[rows])
        m = (dx_[:, None] * ps) @ np.diag(1.0 / py[cols]) @ (ps.T * dx_[None, :])
        m = 0.5 * (m + m.T)
        ev = np.sort(np.linalg.eigvalsh(m))[::-1]
        f[13] = np.sqrt(max(0.0, float(ev[1])))
    else:
        f[13] = 0.0
    return f


def haralick_batch(P: np.ndarray, symmetric: bool) -> np.ndarray:
    """Features of a stack of count matrices (..., N, N) -> (..., 14) float64."""
    P = np.asarray(P)
    flat = P.reshape(-1, P.shape[-2], P.shape[-1])
    S = symmetrize(flat) if symmetric else flat.astype(np.uint64)
    p = normalize(S)
    out = np.stack([haralick(pk) for pk in p]) if len(p) else np.zeros((0, 14))
    return out.reshape(P.shape[:-2] + (14,))


def window_maps(counts: np.ndarray, symmetric: bool = False) -> np.ndarray:
    """Local texture maps from per-window counts (n_win, n_off, N, N).

    Returns (4, n_win, n_off) float64 maps in WINDOW_MAP_NAMES order:
    contrast, angular second moment, inverse difference moment, entropy."""
    C = np.asarray(counts)
    S = symmetrize(C) if symmetric else C.astype(np.uint64)
    p = normalize(S)
    n = p.shape[-1]
    i = np.arange(n, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[None, :]
    contrast = ((i - j) ** 2 * p).sum(axis=(-1, -2))
    asm = (p * p).sum(axis=(-1, -2))
    idm = (p / (1.0 + (i - j) ** 2)).sum(axis=(-1, -2))
    ent = -_plogp(p).sum(axis=(-1, -2))
    return np.stack([contrast, asm, idm, ent])
