"""Pins for the oracle's GLCM counts (Eq. 1), independent of the oracle itself.

Each check comes from the definition or from mathematics the definition
fixes, never from the oracle's own loops: hand-counted images, a pure-Python
enumeration of all pixel pairs, exhaustive tiny images, the closed-form pair
total, the transpose identity for the opposite direction (theta + 180 deg),
constant images, marginals equal to 1-D histograms, a numpy bincount
formulation, and the stripe decomposition with halo rows of Scheme 3
(Eqs. 7-9).  The gray-level histogram is pinned by hand counts, by the GLCM
marginals plus the pixels that anchor no pair, and by enumeration."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_counted.json")


def _brute(img, n, dx, dy, levels_mode):
    """Enumerate every ordered pair of pixel positions and keep those at (dx, dy)."""
    h, w = img.shape
    bits = 8 * img.itemsize
    P = np.zeros((n, n), dtype=np.int64)
    skipped = 0
    pos = [(x, y) for y in range(h) for x in range(w)]
    for (x1, y1) in pos:
        for (x2, y2) in pos:
            if x2 - x1 != dx or y2 - y1 != dy:
                continue
            v1, v2 = int(img[y1, x1]), int(img[y2, x2])
            if levels_mode:
                i, j = v1, v2
            else:
                i, j = (v1 * n) >> bits, (v2 * n) >> bits
            if i >= n or j >= n:
                skipped += 1
                continue
            P[i, j] += 1
    return P, skipped


def test_hand_counted_goldens(oracle_lib):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        img = np.array(c["image"], dtype=np.dtype(c["dtype"]))
        n = c["levels"]
        for key, want in c.get("glcm", {}).items():
            dx, dy = map(int, key.split(","))
            got = oracle.glcm(img, n, [(dx, dy)], levels_mode=c["levels_mode"])[0]
            assert np.array_equal(got, np.array(want)), (c["name"], key)
        for key, entries in c.get("glcm_sparse", {}).items():
            dx, dy = map(int, key.split(","))
            want = np.zeros((n, n), dtype=np.int64)
            for i, j, v in entries:
                want[i, j] += v
            got = oracle.glcm(img, n, [(dx, dy)], levels_mode=c["levels_mode"])[0]
            assert np.array_equal(got, want), (c["name"], key)


def test_exhaustive_2x2_binary(oracle_lib):
    offs = [(dx, dy) for dx in range(-2, 3) for dy in range(-2, 3)]
    for bits in itertools.product([0, 1], repeat=4):
        img = np.array(bits, dtype=np.uint8).reshape(2, 2)
        got = oracle.glcm(img, 2, offs, levels_mode=True)
        for k, (dx, dy) in enumerate(offs):
            want, _ = _brute(img, 2, dx, dy, True)
            assert np.array_equal(got[k], want)


@pytest.mark.parametrize("seed", range(12))
def test_random_tiny_vs_enumeration(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    h, w = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    dtype = np.uint8 if seed % 2 == 0 else np.uint16
    n = int(rng.choice([2, 3, 4, 5, 8, 16]))
    top = 256 if dtype == np.uint8 else 65536
    img = rng.integers(0, top, size=(h, w)).astype(dtype)
    offs = [(int(rng.integers(-4, 5)), int(rng.integers(-4, 5))) for _ in range(5)]
    got = oracle.glcm(img, n, offs)
    for k, (dx, dy) in enumerate(offs):
        want, _ = _brute(img, n, dx, dy, False)
        assert np.array_equal(got[k], want), (h, w, n, dx, dy)


def test_levels_mode_out_of_range_pairs_are_skipped(oracle_lib):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 10, size=(7, 6)).astype(np.uint8)  # some values >= N = 8
    for dx, dy in [(1, 0), (0, -1), (-2, 3)]:
        got, skipped = oracle.glcm(img, 8, [(dx, dy)], levels_mode=True, return_skipped=True)
        want, want_skipped = _brute(img, 8, dx, dy, True)
        assert np.array_equal(got[0], want)
        assert skipped == want_skipped


@pytest.mark.parametrize("w,h", [(1, 1), (5, 3), (64, 17), (300, 200)])
def test_total_closed_form(oracle_lib, w, h):
    img = np.random.default_rng(w * h).integers(0, 256, size=(h, w)).astype(np.uint8)
    offs = [(1, 0), (1, -1), (0, -1), (-1, -1), (4, -4), (-3, 2), (w, 0), (0, h), (w + 2, -1)]
    P = oracle.glcm(img, 16, offs)
    for k, (dx, dy) in enumerate(offs):
        assert int(P[k].sum()) == max(0, w - abs(dx)) * max(0, h - abs(dy))


def test_opposite_direction_is_transpose(oracle_lib):
    img = np.random.default_rng(3).integers(0, 256, size=(37, 53)).astype(np.uint8)
    for dx, dy in [(1, 0), (1, -1), (0, -1), (-1, -1), (4, -2), (3, 5)]:
        a = oracle.glcm(img, 32, [(dx, dy), (-dx, -dy)])
        assert np.array_equal(a[1], a[0].T)


@pytest.mark.parametrize("n", [8, 16, 32, 256])
def test_constant_image_fills_one_bin(oracle_lib, n):
    img = np.full((33, 41), 128, dtype=np.uint8)
    P = oracle.glcm(img, n, [(1, 0), (1, -1), (0, -1), (-1, -1)])
    for k, (dx, dy) in enumerate([(1, 0), (1, -1), (0, -1), (-1, -1)]):
        want = np.zeros((n, n), dtype=np.int64)
        want[n // 2, n // 2] = (41 - abs(dx)) * (33 - abs(dy))
        assert np.array_equal(P[k], want)


def test_marginals_are_histograms(oracle_lib):
    rng = np.random.default_rng(11)
    img = rng.integers(0, 65536, size=(45, 70)).astype(np.uint16)
    n = 32
    q = (img.astype(np.int64) * n) >> 16
    h, w = img.shape
    for dx, dy in [(1, 0), (2, -2), (0, -4), (-3, -1), (-2, 3)]:
        P = oracle.glcm(img, n, [(dx, dy)])[0].astype(np.int64)
        ax0, ax1 = max(0, -dx), w - max(0, dx)
        ay0, ay1 = max(0, -dy), h - max(0, dy)
        anchors = q[ay0:ay1, ax0:ax1]
        partners = q[ay0 + dy:ay1 + dy, ax0 + dx:ax1 + dx]
        assert np.array_equal(P.sum(axis=1), np.bincount(anchors.reshape(-1), minlength=n))
        assert np.array_equal(P.sum(axis=0), np.bincount(partners.reshape(-1), minlength=n))


def test_bincount_formulation_agrees(oracle_lib):
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(257, 389)).astype(np.uint8)
    n = 16
    q = (img.astype(np.int64) * n) >> 8
    h, w = img.shape
    offs = [(1, 0), (1, -1), (0, -1), (-1, -1), (2, 0), (4, -4)]
    P = oracle.glcm(img, n, offs)
    for k, (dx, dy) in enumerate(offs):
        ax0, ax1 = max(0, -dx), w - max(0, dx)
        ay0, ay1 = max(0, -dy), h - max(0, dy)
        i = q[ay0:ay1, ax0:ax1]
        j = q[ay0 + dy:ay1 + dy, ax0 + dx:ax1 + dx]
        want = np.bincount((i * n + j).reshape(-1), minlength=n * n).reshape(n, n)
        assert np.array_equal(P[k], want)


@pytest.mark.parametrize("k_stripes", [2, 3, 7])
def test_stripes_with_halo_sum_to_whole_image(oracle_lib, k_stripes):
    """Scheme 3 (Eqs. 7-9): stripes that own their anchor rows and read the
    partner rows of the halo add up to the whole-image GLCM."""
    rng = np.random.default_rng(k_stripes)
    img = rng.integers(0, 256, size=(61, 47)).astype(np.uint8)
    h = img.shape[0]
    bounds = np.linspace(0, h, k_stripes + 1).astype(int)
    for dx, dy in [(1, 0), (1, -1), (0, -1), (-1, -1), (2, -4), (1, 3)]:
        whole = oracle.glcm(img, 8, [(dx, dy)])[0].astype(np.int64)
        acc = np.zeros_like(whole)
        for r0, r1 in zip(bounds[:-1], bounds[1:]):
            lo = max(0, r0 + min(0, dy))
            hi = min(h, r1 + max(0, dy))
            acc += oracle.glcm(img[lo:hi], 8, [(dx, dy)])[0]
        assert np.array_equal(acc, whole)


def test_empty_when_offset_exceeds_image(oracle_lib):
    img = np.zeros((3, 4), dtype=np.uint8)
    P = oracle.glcm(img, 8, [(4, 0), (0, 3), (-5, -5)])
    assert P.sum() == 0


def test_window_glcm_equals_crop(oracle_lib):
    """A window's local GLCM is the whole-image GLCM of the cropped window."""
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(40, 50)).astype(np.uint8)
    offs = [(1, 0), (1, -1), (0, -1), (-1, -1)]
    win, stride = 15, 4
    W = oracle.window_glcm(img, 16, offs, win, stride)
    nwy, nwx = (40 - win) // stride + 1, (50 - win) // stride + 1
    assert W.shape == (nwy * nwx, 4, 16, 16)
    for idx in [0, 3, nwx, nwy * nwx - 1]:
        wy, wx = divmod(idx, nwx)
        crop = img[wy * stride:wy * stride + win, wx * stride:wx * stride + win]
        assert np.array_equal(W[idx], oracle.glcm(crop, 16, offs))
    for k, (dx, dy) in enumerate(offs):
        assert int(W[0, k].sum()) == (win - abs(dx)) * (win - abs(dy))


# ---- the gray-level histogram (one-pixel statistic, Sec. I) ----------------

def test_histogram_hand_counted(oracle_lib):
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    n_checked = 0
    for c in cases:
        if "histogram" not in c:
            continue
        img = np.array(c["image"], dtype=np.dtype(c["dtype"]))
        got = oracle.histogram(img, c["levels"], levels_mode=c["levels_mode"])
        assert np.array_equal(got, np.array(c["histogram"])), c["name"]
        n_checked += 1
    assert n_checked == 3


@pytest.mark.parametrize("seed", range(4))
def test_histogram_is_glcm_marginal_plus_last_column(oracle_lib, seed):
    """Every pixel but those of the last column is the anchor of exactly one
    (1, 0) pair, so the histogram is the row sums of P(1, 0) plus the levels
    of the last column; likewise the column sums of P(0, 1) plus the first
    row's levels."""
    rng = np.random.default_rng(400 + seed)
    h, w = int(rng.integers(1, 30)), int(rng.integers(2, 40))
    dt = np.uint8 if seed % 2 == 0 else np.uint16
    img = rng.integers(0, np.iinfo(dt).max + 1, size=(h, w)).astype(dt)
    n = [2, 7, 16, 256][seed]
    bits = 8 * img.itemsize
    hist = oracle.histogram(img, n)
    last = [(int(v) * n) >> bits for v in img[:, -1]]
    want = oracle.glcm(img, n, [(1, 0)])[0].sum(axis=1).astype(np.int64)
    for q in last:
        want[q] += 1
    assert np.array_equal(hist, want)
    first_row = [(int(v) * n) >> bits for v in img[0, :]]
    want2 = oracle.glcm(img, n, [(0, 1)])[0].sum(axis=0).astype(np.int64)
    for q in first_row:
        want2[q] += 1
    assert np.array_equal(hist, want2)
    assert int(hist.sum()) == h * w


def test_histogram_brute_force_and_levels_mode(oracle_lib):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 12, size=(9, 11)).astype(np.uint8)
    n = 10
    want = np.zeros(n, dtype=np.int64)
    skipped = 0
    for y in range(img.shape[0]):
        for x in range(img.shape[1]):
            v = int(img[y, x])
            if v >= n:
                skipped += 1
            else:
                want[v] += 1
    got, s = oracle.histogram(img, n, levels_mode=True, return_skipped=True)
    assert np.array_equal(got, want) and s == skipped and skipped > 0
    const = np.full((5, 6), 200, dtype=np.uint8)
    hc = oracle.histogram(const, 8)
    assert hc[(200 * 8) >> 8] == 30 and hc.sum() == 30


# ---- flat-wrap mode (Eq. 2 read literally on the row-major buffer) ----------

def _flat_brute(img, n, dx, dy):
    """Pure-Python enumeration of the flat buffer: pixel p pairs with p + dy W + dx."""
    h, w = img.shape
    flat = [int(v) for v in img.reshape(-1)]
    P = np.zeros((n, n), dtype=np.uint32)
    off = dy * w + dx
    for p in range(h * w):
        q = p + off
        if 0 <= q < h * w:
            P[flat[p], flat[q]] += 1
    return P


def test_flat_hand_worked_3x4():
    # Pixels 0..11 row-major in a 4-wide image, levels as given.  Offset (1, 0)
    # pairs p with p + 1: eleven pairs, two of them across row ends (3 -> 4 and
    # 7 -> 8), which the no-wrap counts leave out.  Offset (1, -1) (45 deg)
    # pairs p with p - 3: nine pairs, p = 3..11; (3 -> 0), (7 -> 4) and
    # (11 -> 8) wrap (their partner is the first pixel of the same row).
    img = np.arange(12, dtype=np.uint8).reshape(3, 4)
    P = oracle.glcm_flat(img, 12, [(1, 0), (1, -1)], levels_mode=True)
    want0 = np.zeros((12, 12), np.uint32)
    for p in range(11):
        want0[p, p + 1] = 1
    want1 = np.zeros((12, 12), np.uint32)
    for p in range(3, 12):
        want1[p, p - 3] = 1
    assert np.array_equal(P[0], want0) and np.array_equal(P[1], want1)
    nowrap = oracle.glcm(img, 12, [(1, 0), (1, -1)], levels_mode=True)
    assert int(nowrap[0].sum()) == 9 and int(nowrap[1].sum()) == 6
    assert P[0][3, 4] == 1 and nowrap[0][3, 4] == 0


@pytest.mark.parametrize("seed", range(12))
def test_flat_matches_brute_force(seed):
    rng = np.random.default_rng(900 + seed)
    h, w, n = int(rng.integers(1, 7)), int(rng.integers(1, 7)), int(rng.integers(2, 6))
    img = rng.integers(0, n, size=(h, w)).astype(np.uint8)
    offs = [(int(rng.integers(-8, 9)), int(rng.integers(-3, 4))) for _ in range(6)] + [(1, 0), (-1, -1), (w, 0)]
    P = oracle.glcm_flat(img, n, offs, levels_mode=True)
    for k, (dx, dy) in enumerate(offs):
        assert np.array_equal(P[k], _flat_brute(img, n, dx, dy)), (h, w, dx, dy)


@pytest.mark.parametrize("seed", range(6))
def test_flat_is_the_lagged_pair_histogram_of_the_raveled_image(seed):
    """The flat GLCM is the joint histogram of (s[t], s[t + L]) over the raveled
    levels s at lag L = dy W + dx, formed here by numpy bincount; its total is
    W H - |L|, and lag -L gives the transpose."""
    rng = np.random.default_rng(950 + seed)
    h, w, n = int(rng.integers(2, 40)), int(rng.integers(2, 40)), 16
    img = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    s = (img.astype(np.int64) * n) >> 8
    s = s.reshape(-1)
    for dx, dy in [(1, 0), (1, -1), (0, -1), (-1, -1), (3, 2), (w + 2, -1)]:
        L = dy * w + dx
        if abs(L) >= h * w:
            continue
        a, b = (s[:-L], s[L:]) if L > 0 else ((s[-L:], s[:L]) if L < 0 else (s, s))
        want = np.bincount(a * n + b, minlength=n * n).reshape(n, n)
        P = oracle.glcm_flat(img, n, [(dx, dy), (-dx, -dy)])
        assert np.array_equal(P[0], want.astype(np.uint32)), (dx, dy)
        assert int(P[0].sum()) == h * w - abs(L)
        assert np.array_equal(P[1], P[0].T)


def test_flat_equals_no_wrap_plus_row_seams():
    """Flat counts = the in-bounds (no-wrap) counts + the pairs whose partner
    column x + dx leaves [0, W) (enumerated here from the seam columns only)."""
    rng = np.random.default_rng(77)
    img = rng.integers(0, 256, size=(33, 29)).astype(np.uint8)
    h, w, n = img.shape[0], img.shape[1], 8
    q = (img.astype(np.int64) * n) >> 8
    for dx, dy in [(1, 0), (2, -1), (-3, -2), (4, 1)]:
        seam = np.zeros((n, n), np.int64)
        xs = range(w - dx, w) if dx > 0 else range(0, -dx)
        for y in range(h):
            for x in xs:
                p2 = (y + dy) * w + x + dx
                if 0 <= p2 < h * w:
                    seam[q[y, x], q[p2 // w, p2 % w]] += 1
        nowrap = oracle.glcm(img, n, [(dx, dy)])[0].astype(np.int64)
        assert np.array_equal(oracle.glcm_flat(img, n, [(dx, dy)])[0].astype(np.int64), nowrap + seam), (dx, dy)
