"""Pins for the float64 Haralick oracle against closed forms and identities.

None of these re-types the oracle's formulas: each expected value is either
a closed form for a constructed matrix (uniform, one-hot, diagonal,
independent, block-diagonal, 2 x 2 tables where correlation is the phi
coefficient and the maximal correlation is its magnitude) or an identity of
information theory (HXY1 = HXY2 = HX + HY, so f12 and f13 are functions of
the mutual information) or of probability (f4 is the variance of the row
marginal; f7/f10 are variances of the sum/difference distributions)."""
import math

import numpy as np
import pytest

import oracle
from oracle import haralick

TOL = 1e-12


@pytest.mark.parametrize("n", [2, 3, 8, 32])
def test_uniform(n):
    p = np.full((n, n), 1.0 / (n * n))
    f = haralick(p)
    assert f[0] == pytest.approx(1.0 / n ** 2, abs=TOL)
    assert f[1] == pytest.approx((n * n - 1) / 6.0, rel=TOL)
    assert f[2] == pytest.approx(0.0, abs=1e-10)
    assert f[3] == pytest.approx((n * n - 1) / 12.0, rel=TOL)
    assert f[5] == pytest.approx(n - 1.0, rel=TOL)
    assert f[8] == pytest.approx(2 * math.log(n), rel=TOL)
    assert f[11] == pytest.approx(0.0, abs=1e-10)
    assert f[12] == pytest.approx(0.0, abs=1e-6)
    assert f[13] == pytest.approx(0.0, abs=1e-6)


@pytest.mark.parametrize("a", [0, 3, 7])
def test_one_hot(a):
    p = np.zeros((8, 8))
    p[a, a] = 1.0
    f = haralick(p)
    assert f[0] == 1.0 and f[1] == 0.0 and f[4] == 1.0 and f[8] == 0.0
    assert f[5] == pytest.approx(2 * a)
    assert f[6] == 0.0 and f[7] == 0.0 and f[9] == 0.0 and f[10] == 0.0
    assert f[2] == 1.0  # degenerate (zero variance) correlation is defined as 1
    assert f[13] == 0.0  # only one row in the support


def _idm_uniform(n):
    """Inverse difference moment of the uniform n x n distribution, counted by
    diagonals: n cells have |i - j| = 0 and 2 (n - k) cells have |i - j| = k."""
    return (n + sum(2.0 * (n - k) / (1.0 + k * k) for k in range(1, n))) / (n * n)


@pytest.mark.parametrize("n", [3, 4, 8, 32])
def test_idm_uniform_by_diagonals(n):
    p = np.full((n, n), 1.0 / (n * n))
    assert haralick(p)[4] == pytest.approx(_idm_uniform(n), rel=TOL)


def test_idm_hand_worked_3x3():
    # Half the mass at (0, 2) (|i - j| = 2, weight 1/5), a quarter at (1, 1)
    # (weight 1) and a quarter at (2, 1) (|i - j| = 1, weight 1/2):
    # 0.5 / 5 + 0.25 + 0.25 / 2 = 0.475.
    p = np.zeros((3, 3))
    p[0, 2], p[1, 1], p[2, 1] = 0.5, 0.25, 0.25
    assert haralick(p)[4] == pytest.approx(0.475, rel=TOL)


@pytest.mark.parametrize("n", [2, 5, 16])
def test_diagonal(n):
    p = np.eye(n) / n
    f = haralick(p)
    assert f[2] == pytest.approx(1.0, abs=TOL)
    assert f[13] == pytest.approx(1.0, abs=1e-9)
    assert f[12] == pytest.approx(math.sqrt(1 - 1.0 / n ** 2), rel=1e-12)
    assert f[1] == 0.0
    assert f[8] == pytest.approx(math.log(n), rel=TOL)
    assert f[11] == pytest.approx(-1.0, rel=1e-12)  # -I / max(HX, HY) = -ln n / ln n


def test_independent_product():
    rng = np.random.default_rng(1)
    px = rng.random(12); px /= px.sum()
    py = rng.random(12); py /= py.sum()
    f = haralick(np.outer(px, py))
    assert abs(f[11]) < 1e-12
    assert abs(f[12]) < 1e-6
    assert abs(f[13]) < 1e-6


def test_block_diagonal_has_unit_second_correlation():
    rng = np.random.default_rng(2)
    p = np.zeros((6, 6))
    p[:3, :3] = rng.random((3, 3))
    p[3:, 3:] = rng.random((3, 3))
    p /= p.sum()
    assert haralick(p)[13] == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_2x2_closed_forms(seed):
    a, b, c, d = np.random.default_rng(seed).random(4) + 0.05
    s = a + b + c + d
    a, b, c, d = a / s, b / s, c / s, d / s
    p = np.array([[a, b], [c, d]])
    f = haralick(p)
    r0, r1, c0, c1 = a + b, c + d, a + c, b + d
    phi = (a * d - b * c) / math.sqrt(r0 * r1 * c0 * c1)
    assert f[0] == pytest.approx(a * a + b * b + c * c + d * d, rel=TOL)
    assert f[1] == pytest.approx(b + c, rel=TOL)
    assert f[2] == pytest.approx(phi, abs=1e-12)
    assert f[3] == pytest.approx(r0 * r1, rel=1e-12)
    assert f[4] == pytest.approx(a + d + (b + c) / 2, rel=TOL)
    assert f[5] == pytest.approx((b + c) + 2 * d, rel=TOL)
    mean_s = (b + c) + 2 * d
    assert f[6] == pytest.approx(a * mean_s ** 2 + (b + c) * (1 - mean_s) ** 2 + d * (2 - mean_s) ** 2, rel=1e-12)
    assert f[9] == pytest.approx((b + c) * (a + d), rel=1e-12)
    assert f[10] == pytest.approx(-((b + c) * math.log(b + c) + (a + d) * math.log(a + d)), rel=1e-12)
    assert f[13] == pytest.approx(abs(phi), abs=1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_information_identities(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 12))
    p = rng.random((n, n)) ** 3
    p[rng.random((n, n)) < 0.2] = 0.0
    p /= p.sum()
    f = haralick(p)
    px, py = p.sum(1), p.sum(0)
    nz = p > 0
    mi = float((p[nz] * np.log(p[nz] / np.outer(px, py)[nz])).sum())
    hx = -float((px[px > 0] * np.log(px[px > 0])).sum())
    hy = -float((py[py > 0] * np.log(py[py > 0])).sum())
    assert f[11] == pytest.approx(-mi / max(hx, hy), abs=1e-12)
    assert f[12] == pytest.approx(math.sqrt(1 - math.exp(-2 * mi)), abs=1e-9)
    lv = np.arange(n)
    mux = (lv * px).sum()
    assert f[3] == pytest.approx(((lv - mux) ** 2 * px).sum(), rel=1e-12)
    # f14 is the second singular value of D_x^-1/2 P D_y^-1/2 (restricted to the support).
    r, c = px > 0, py > 0
    A = p[np.ix_(r, c)] / np.sqrt(np.outer(px[r], py[c]))
    sv = np.linalg.svd(A, compute_uv=False)
    assert f[13] == pytest.approx(sv[1] if len(sv) > 1 else 0.0, abs=1e-9)


def test_transpose_invariance():
    rng = np.random.default_rng(4)
    p = rng.random((9, 9)); p /= p.sum()
    f, g = haralick(p), haralick(p.T)
    for k in [0, 1, 2, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13]:
        assert f[k] == pytest.approx(g[k], rel=1e-10, abs=1e-12)


def test_entropy_of_uniform_support():
    p = np.zeros((8, 8))
    cells = [(0, 1), (2, 5), (7, 7), (3, 3), (6, 0)]
    for c in cells:
        p[c] = 1.0 / len(cells)
    assert haralick(p)[8] == pytest.approx(math.log(len(cells)), rel=TOL)


def test_empty_glcm_gives_zero_features():
    assert np.all(haralick(np.zeros((4, 4))) == 0)
    assert np.all(oracle.normalize(np.zeros((4, 4), dtype=np.uint32)) == 0)


def test_symmetrize_normalize_totals():
    P = np.random.default_rng(0).integers(0, 1000, size=(3, 16, 16)).astype(np.uint32)
    S = oracle.symmetrize(P)
    assert np.array_equal(S.sum(axis=(1, 2)), 2 * P.astype(np.uint64).sum(axis=(1, 2)))
    assert np.array_equal(S, np.swapaxes(S, 1, 2))
    p = oracle.normalize(S)
    assert np.allclose(p.sum(axis=(1, 2)), 1.0, rtol=0, atol=1e-15)


def test_window_maps_match_full_features():
    rng = np.random.default_rng(8)
    C = rng.integers(0, 50, size=(5, 4, 16, 16)).astype(np.uint32)
    maps = oracle.window_maps(C)
    feats = oracle.haralick_batch(C, symmetric=False)
    assert np.allclose(maps[0], feats[..., 1], rtol=1e-14)
    assert np.allclose(maps[1], feats[..., 0], rtol=1e-14)
    assert np.allclose(maps[2], feats[..., 4], rtol=1e-14)
    assert np.allclose(maps[3], feats[..., 8], rtol=1e-14)


@pytest.mark.parametrize("n", [3, 16])
def test_window_maps_closed_forms(n):
    """Window maps of constructed count tables: uniform counts (contrast
    (n^2 - 1) / 6, ASM 1 / n^2, IDM counted by diagonals, entropy 2 ln n), a
    single bin (0, 0, 1, 0), and the hand-worked 3 x 3 table of
    test_idm_hand_worked_3x3 scaled to counts 2 : 1 : 1."""
    C = np.zeros((3, 1, n, n), dtype=np.uint32)
    C[0, 0] = 7
    C[1, 0, n - 1, n - 1] = 5
    C[2, 0, 0, 2], C[2, 0, 1, 1], C[2, 0, 2, 1] = 2, 1, 1
    m = oracle.window_maps(C)
    assert m[0, 0, 0] == pytest.approx((n * n - 1) / 6.0, rel=TOL)
    assert m[1, 0, 0] == pytest.approx(1.0 / (n * n), rel=TOL)
    assert m[2, 0, 0] == pytest.approx(_idm_uniform(n), rel=TOL)
    assert m[3, 0, 0] == pytest.approx(2 * math.log(n), rel=TOL)
    assert (m[0, 1, 0], m[1, 1, 0], m[2, 1, 0], m[3, 1, 0]) == (0.0, 1.0, 1.0, 0.0)
    assert m[0, 2, 0] == pytest.approx(0.5 * 4 + 0.25 * 1, rel=TOL)
    assert m[1, 2, 0] == pytest.approx(0.25 + 0.0625 + 0.0625, rel=TOL)
    assert m[2, 2, 0] == pytest.approx(0.475, rel=TOL)
    assert m[3, 2, 0] == pytest.approx(-(0.5 * math.log(0.5) + 0.5 * math.log(0.25)), rel=TOL)


@pytest.mark.parametrize("seed", range(8))
def test_moment_identities(seed):
    """Features of the sum / difference distributions and the correlation
    checked through moments of the joint distribution of (i, j):
    f6 = E[i + j], f7 = Var(i) + Var(j) + 2 Cov(i, j), f2 = E[(i - j)^2],
    f10 = E[(i - j)^2] - E[|i - j|]^2, f3 = Cov / (sd_i sd_j) from np.cov with
    the cells' probabilities as weights, and f8 / f11 the entropies of the
    distributions of i + j and |i - j| formed by bincount."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(3, 21))
    p = rng.random((n, n)) ** 2
    p[rng.random((n, n)) < 0.3] = 0.0
    p[rng.integers(n), rng.integers(n)] += 0.5
    p /= p.sum()
    f = haralick(p)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    w = p.ravel()
    i, j = ii.ravel().astype(float), jj.ravel().astype(float)
    cov = np.cov(np.stack([i, j]), aweights=w, ddof=0)
    ei, ej = float((w * i).sum()), float((w * j).sum())
    assert f[5] == pytest.approx(ei + ej, rel=1e-12)
    assert f[6] == pytest.approx(cov[0, 0] + cov[1, 1] + 2 * cov[0, 1], rel=1e-10)
    e2 = float((w * (i - j) ** 2).sum())
    assert f[1] == pytest.approx(e2, rel=1e-12)
    assert f[9] == pytest.approx(e2 - float((w * np.abs(i - j)).sum()) ** 2, rel=1e-9, abs=1e-12)
    assert f[2] == pytest.approx(cov[0, 1] / math.sqrt(cov[0, 0] * cov[1, 1]), abs=1e-10)

    def ent(q):
        q = q[q > 0]
        return -float((q * np.log(q)).sum())

    assert f[7] == pytest.approx(ent(np.bincount((i + j).astype(int), weights=w)), rel=1e-12)
    assert f[10] == pytest.approx(ent(np.bincount(np.abs(i - j).astype(int), weights=w)), rel=1e-12)
    pd = np.bincount(np.abs(i - j).astype(int), weights=w)
    assert f[4] == pytest.approx(float((pd / (1.0 + np.arange(len(pd)) ** 2)).sum()), rel=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_library_routines_on_count_tables(seed):
    """Features of integer count tables against library routines that compute
    the same quantities by their own code: scikit-learn's mutual information
    of a contingency table (f12, f13), scipy's entropy (f8, f9, f11), scipy's
    Pearson correlation of the expanded (i, j) samples (f3), and numpy's
    variance of the expanded samples (f4, f7)."""
    pytest.importorskip("sklearn")
    from scipy import stats
    from sklearn.metrics import mutual_info_score

    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 17))
    C = rng.integers(0, 9, size=(n, n))
    C[rng.random((n, n)) < 0.35] = 0
    C[0, n - 1] += 3
    C[n - 1, 0] += 2
    p = C / C.sum()
    f = haralick(p)
    ii, jj = np.nonzero(C)
    reps = C[ii, jj]
    si, sj = np.repeat(ii, reps).astype(float), np.repeat(jj, reps).astype(float)
    mi = mutual_info_score(None, None, contingency=C)
    hx, hy = stats.entropy(C.sum(1)), stats.entropy(C.sum(0))
    assert f[11] == pytest.approx(-mi / max(hx, hy), abs=1e-10)
    assert f[12] == pytest.approx(math.sqrt(max(0.0, 1 - math.exp(-2 * mi))), abs=1e-8)
    assert f[8] == pytest.approx(stats.entropy(C.ravel()), rel=1e-12)
    assert f[7] == pytest.approx(stats.entropy(np.bincount((si + sj).astype(int))), rel=1e-12)
    assert f[10] == pytest.approx(stats.entropy(np.bincount(np.abs(si - sj).astype(int))), rel=1e-12)
    assert f[2] == pytest.approx(stats.pearsonr(si, sj).statistic, abs=1e-10)
    assert f[3] == pytest.approx(np.var(si), rel=1e-12)
    assert f[6] == pytest.approx(np.var(si + sj), rel=1e-10)
    assert f[4] == pytest.approx(float(np.mean(1.0 / (1.0 + (si - sj) ** 2))), rel=1e-12)
