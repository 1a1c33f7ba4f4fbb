"""Seeded synthetic inputs for the GLCM workloads.

This module only makes input bytes (images, offset lists, request streams).
It holds none of the co-occurrence arithmetic: no quantization, no pairing,
no voting, no features.  Both the CUDA path (through the tests and the
bench) and the CPU oracle consume exactly the bytes produced here, so parity
does not depend on how the images are made.

Recipes (all deterministic from the seed):

* ``iid``      -- ``numpy.random.default_rng(seed).integers(lo, hi)`` over the
                  full range of the pixel type (or a given range).
* ``smooth``   -- float64 N(0, 1) noise from ``default_rng(seed)``, blurred by a
                  circular (periodic-boundary) Gaussian of standard deviation
                  ``sigma`` pixels applied in the Fourier domain, min-max
                  rescaled to the full range of the pixel type and rounded
                  with ``numpy.rint``.  This stands in for the paper's
                  slowly varying photograph, Fig. 1(a).
* ``constant`` -- every pixel equal to one value (128 for uint8).

The paper's two test photographs (Fig. 1) are not available; the iid images
stand in for Fig. 1(b) (drastic gray-level changes) and the smooth images for
Fig. 1(a) (small changes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20171018

# Offsets as (dx, dy); the partner of anchor (x, y) is (x + dx, y + dy) with
# y the row index growing downwards.  Distance d at 0/45/90/135 degrees.
ANGLES = (0, 45, 90, 135)


def angle_offset(d: int, theta: int) -> tuple[int, int]:
    """(dx, dy) for distance d at angle theta, chessboard steps on diagonals."""
    table = {0: (d, 0), 45: (d, -d), 90: (0, -d), 135: (-d, -d)}
    return table[theta]


def offsets_for(distances, angles=ANGLES) -> list[tuple[int, int]]:
    return [angle_offset(d, t) for d in distances for t in angles]


def iid(seed: int, h: int, w: int, dtype=np.uint8, lo: int = 0, hi: int | None = None) -> np.ndarray:
    dt = np.dtype(dtype)
    if hi is None:
        hi = int(np.iinfo(dt).max) + 1
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=(h, w), dtype=np.int64).astype(dt)


def _gauss_blur_periodic(x: np.ndarray, sigma: float) -> np.ndarray:
    h, w = x.shape
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    g = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * (fy * fy + fx * fx))
    return np.fft.irfft2(np.fft.rfft2(x) * g, s=(h, w))


def smooth(seed: int, h: int, w: int, sigma: float, dtype=np.uint8) -> np.ndarray:
    dt = np.dtype(dtype)
    top = float(np.iinfo(dt).max)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((h, w))
    b = _gauss_blur_periodic(noise, sigma)
    lo, hi = float(b.min()), float(b.max())
    if hi <= lo:
        return np.zeros((h, w), dtype=dt)
    y = np.rint((b - lo) * (top / (hi - lo)))
    return np.clip(y, 0, top).astype(dt)


def constant(h: int, w: int, value: int = 128, dtype=np.uint8) -> np.ndarray:
    return np.full((h, w), value, dtype=np.dtype(dtype))


def image(kind: str, seed: int, h: int, w: int, dtype=np.uint8, sigma: float = 8.0) -> np.ndarray:
    if kind == "iid":
        return iid(seed, h, w, dtype)
    if kind == "smooth":
        return smooth(seed, h, w, sigma, dtype)
    if kind == "constant":
        top = int(np.iinfo(np.dtype(dtype)).max)
        return constant(h, w, (top + 1) // 2, dtype)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# Workload recipes, one per configuration.
# ---------------------------------------------------------------------------

def plain_512():
    """One 512x512 uint8 image of levels in [0, 8), N = 8, offset (1, 0)."""
    img = iid(BASE_SEED + 1, 512, 512, np.uint8, 0, 8)
    return img, 8, [(1, 0)]


CONTENTION_LEVELS = (8, 16, 32, 256)
CONTENTION_KINDS = ("iid", "smooth", "constant")
CONTENTION_OFFSETS = [(1, 0), (1, -1), (0, -1), (-1, -1)]


def contention_jobs(side: int = 4096, levels=CONTENTION_LEVELS, kinds=CONTENTION_KINDS, sigma: float = 8.0):
    """Contention sweep: one distinct image per (kind, N) pair, 4 offsets at d = 1.

    Returns a list of dicts {kind, levels, image, offsets}.  Each (kind, N)
    gets its own seed so that the batch holds distinct bytes (larger than L2
    at 4096^2 x 12 images)."""
    jobs = []
    for ki, kind in enumerate(kinds):
        for li, n in enumerate(levels):
            seed = BASE_SEED + 100 + 10 * ki + li
            img = image(kind, seed, side, side, np.uint8, sigma)
            jobs.append(dict(kind=kind, levels=n, image=img, offsets=list(CONTENTION_OFFSETS)))
    return jobs


def multispectral_band(b: int, side: int = 8192, n_bands: int = 8, sigma: float = 16.0) -> np.ndarray:
    """Band b of the multispectral stack: iid over 0..65535 for the first
    half of the bands, smooth (sigma px) for the rest."""
    seed = BASE_SEED + 200 + b
    if b < n_bands // 2:
        return iid(seed, side, side, np.uint16)
    return smooth(seed, side, side, sigma, np.uint16)


def multispectral_bands(side: int = 8192, n_bands: int = 8, sigma: float = 16.0):
    """8 uint16 bands: 0-3 iid over 0..65535, 4-7 smooth (sigma px)."""
    return [multispectral_band(b, side, n_bands, sigma) for b in range(n_bands)]


MULTISPECTRAL_OFFSETS = offsets_for((1, 2, 4))


def window_image(side: int = 2048, sigma: float = 4.0):
    return smooth(BASE_SEED + 300, side, side, sigma, np.uint8)


def uneven_batch(n_images: int = 1000, lo: int = 64, hi: int = 2048, seed: int = BASE_SEED + 400):
    """Square uint8 images, side = round(exp(U(ln lo, ln hi))), N ~ U{8,16,32},
    iid/smooth alternating by a fair coin, offsets d = 1 x 4 angles."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_images):
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n = int(rng.choice([8, 16, 32]))
        kind = "iid" if rng.random() < 0.5 else "smooth"
        out.append(dict(side=side, levels=n, kind=kind, seed=seed + 1 + k, offsets=list(CONTENTION_OFFSETS)))
    return out


def materialize(job: dict, sigma: float = 8.0) -> np.ndarray:
    return image(job["kind"], job["seed"], job["side"], job["side"], np.uint8, sigma)


@dataclass
class Request:
    rid: int
    arrival_s: float
    side: int
    levels: int
    kind: str
    seed: int
    offsets: list = field(default_factory=list)


def request_stream(n: int, rate_per_s: float, lo: int = 256, hi: int = 8192, seed: int = BASE_SEED + 500):
    """Poisson arrivals at ``rate_per_s``; sides log-uniform in [lo, hi];
    N ~ U{8,16,32,64}; k ~ U{1..12} offsets drawn without replacement from
    d in {1,2,4} x 4 angles; iid/smooth 50/50."""
    rng = np.random.default_rng(seed)
    pool = offsets_for((1, 2, 4))
    t = 0.0
    out = []
    for r in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        n_lv = int(rng.choice([8, 16, 32, 64]))
        k = int(rng.integers(1, 13))
        idx = rng.choice(len(pool), size=k, replace=False)
        offs = [pool[i] for i in sorted(idx)]
        kind = "iid" if rng.random() < 0.5 else "smooth"
        out.append(Request(r, t, side, n_lv, kind, seed + 1 + r, offs))
    return out


SERVE_BASE_SIDE = 8192


def request_crops(reqs, base_side: int = SERVE_BASE_SIDE, seed: int = BASE_SEED + 650):
    """Top-left corner (y0, x0) of each request's side x side window inside a
    base_side^2 image of its kind, uniform over the valid positions.  A
    served request's pixels are that window of one of two base images
    (``image(kind, serve_base_seed(kind), base_side, base_side)``)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in reqs:
        span = base_side - r.side + 1
        out.append((int(rng.integers(0, span)), int(rng.integers(0, span))))
    return out


def serve_base_seed(kind: str) -> int:
    return BASE_SEED + 600 + ("iid", "smooth").index(kind)

