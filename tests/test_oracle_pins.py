"""Pins for the FP64 oracle: closed forms, invariants, library routines and
brute force on tiny inputs.  Each test fixes a part of the oracle with
something other than the oracle itself, so that a dropped term, a wrong sign,
a wrong index or a transposed operand fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest
import scipy.stats

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _single(orc, img, mask, ndim=2, **kw):
    t = orc.extract(img, mask, ndim, **kw)
    return {k: v[0] for k, v in t.items()}


# --------------------------------------------------------------------------
# ROI separation: counts, bounding boxes, min/max (brute force with NumPy)

def test_roi_geometry_bruteforce(orc):
    rng = np.random.default_rng(1)
    mask = rng.integers(0, 5, size=(13, 17)).astype(np.int32)
    mask[mask == 3] = 1000  # sparse label value
    img = rng.integers(0, 65536, size=mask.shape).astype(np.uint16)
    t = orc.extract(img, mask, 2, ng=4)
    labels = np.unique(mask[mask > 0])
    assert list(t["LABEL"]) == list(labels)
    for i, lab in enumerate(labels):
        ys, xs = np.nonzero(mask == lab)
        assert t["AREA"][i] == len(xs)
        assert t["BBOX_XMIN"][i] == xs.min() and t["BBOX_YMIN"][i] == ys.min()
        assert t["BBOX_WIDTH"][i] == xs.max() - xs.min() + 1
        assert t["BBOX_HEIGHT"][i] == ys.max() - ys.min() + 1
        vals = img[mask == lab].astype(np.float64)
        assert t["MIN"][i] == vals.min() and t["MAX"][i] == vals.max()
        assert t["CENTROID_X"][i] == pytest.approx(xs.mean(), rel=1e-15)
        assert t["CENTROID_Y"][i] == pytest.approx(ys.mean(), rel=1e-15)


def test_batch_keys_and_3d_geometry(orc):
    rng = np.random.default_rng(2)
    mask = rng.integers(0, 3, size=(2, 3, 5, 6)).astype(np.int32)
    img = rng.integers(-1000, 3000, size=mask.shape).astype(np.int16)
    t = orc.extract(img, mask, 3, ng=8)
    keys = sorted({(b, l) for b in range(2) for l in np.unique(mask[b]) if l > 0})
    assert list(zip(t["IMAGE"].astype(int), t["LABEL"].astype(int))) == keys
    for i, (b, l) in enumerate(keys):
        zs, ys, xs = np.nonzero(mask[b] == l)
        assert t["AREA"][i] == len(zs)
        assert (t["BBOX_ZMIN"][i], t["BBOX_DEPTH"][i]) == (zs.min(), zs.max() - zs.min() + 1)
        assert t["CENTROID_Z"][i] == pytest.approx(zs.mean(), rel=1e-15)


# --------------------------------------------------------------------------
# Binning (IBSI fixed bin number): equal-width bins over [min, max] with the maximum in the
# last bin; numpy.histogram implements the same equal-width partition.

@pytest.mark.parametrize("lo,hi,n", [(0, 65535, 256), (17, 4000, 32), (100, 103, 8), (5, 5 + 256 * 7, 256),
                                     (0, 64, 64), (30000, 30001, 2)])
def test_binning_vs_numpy_histogram(orc, lo, hi, n):
    vals = np.arange(lo, hi + 1, dtype=np.int64)
    img = vals.astype(np.uint16).reshape(1, -1)
    mask = np.ones_like(img, dtype=np.int32)
    b = orc.roi_bins(img, mask, 2, orc.roi_key(0, 1), n)
    ref, _ = np.histogram(vals, bins=n, range=(lo, hi))
    assert np.array_equal(np.bincount(b, minlength=n), ref)
    assert np.all(np.diff(b) >= 0) and b[0] == 0 and b[-1] == n - 1


def test_binning_exact_width_when_range_is_multiple(orc):
    # range = k*n: every bin holds k values, the top bin one more (the max)
    n, k, lo = 16, 5, 200
    vals = np.arange(lo, lo + k * n + 1, dtype=np.int64)
    img = vals.astype(np.uint16).reshape(1, -1)
    b = orc.roi_bins(img, np.ones_like(img, dtype=np.int32), 2, orc.roi_key(0, 1), n)
    cnt = np.bincount(b, minlength=n)
    assert np.all(cnt[:-1] == k) and cnt[-1] == k + 1


def test_binning_float_and_signed(orc):
    rng = np.random.default_rng(3)
    f = rng.normal(size=500).astype(np.float32).reshape(1, -1)
    b = orc.roi_bins(f, np.ones_like(f, dtype=np.int32), 2, orc.roi_key(0, 1), 64)
    ref, _ = np.histogram(f.astype(np.float64), bins=64, range=(float(f.min()), float(f.max())))
    assert np.array_equal(np.bincount(b, minlength=64), ref)
    s = np.arange(-1000, 3001, 7, dtype=np.int16).reshape(1, -1)
    b = orc.roi_bins(s, np.ones_like(s, dtype=np.int32), 2, orc.roi_key(0, 1), 64)
    ref, _ = np.histogram(s.astype(np.int64), bins=64, range=(-1000, int(s.max())))
    assert np.array_equal(np.bincount(b, minlength=64), ref)


def test_binning_constant_roi_is_bin_zero(orc):
    img = np.full((3, 3), 777, dtype=np.uint16)
    b = orc.roi_bins(img, np.ones_like(img, dtype=np.int32), 2, orc.roi_key(0, 1), 32)
    assert np.all(b == 0)


# --------------------------------------------------------------------------
# GLCM counts: independent NumPy brute force (array shifts), bit-exact

def _np_bins(vals, n):
    lo, hi = vals.min(), vals.max()
    if lo == hi:
        return np.zeros_like(vals, dtype=np.int64)
    h = np.histogram(vals, bins=n, range=(lo, hi))
    edges = h[1]
    return np.clip(np.searchsorted(edges, vals, side="right") - 1, 0, n - 1)


def _np_glcm(img, mask, label, ng, dx, dy, dz=0):
    """Brute-force symmetric GLCM by shifting arrays (z, y, x layout)."""
    img3 = img.reshape((-1,) + img.shape[-2:]) if img.ndim >= 3 else img[None]
    m3 = mask.reshape(img3.shape) if mask.ndim >= 3 else mask[None]
    inroi = m3 == label
    vals = img3[inroi].astype(np.float64)
    bins = np.full(img3.shape, -1, dtype=np.int64)
    bins[inroi] = _np_bins(vals, ng)
    P = np.zeros((ng, ng), dtype=np.int64)
    Z, Y, X = img3.shape
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                if not inroi[z, y, x]:
                    continue
                zz, yy, xx = z + dz, y + dy, x + dx
                if 0 <= zz < Z and 0 <= yy < Y and 0 <= xx < X and inroi[zz, yy, xx]:
                    P[bins[z, y, x], bins[zz, yy, xx]] += 1
                    P[bins[zz, yy, xx], bins[z, y, x]] += 1
    return P


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_glcm_counts_bruteforce_2d(orc, seed):
    rng = np.random.default_rng(10 + seed)
    img = rng.integers(0, 50, size=(8, 8)).astype(np.uint16)
    mask = (rng.random((8, 8)) < 0.7).astype(np.int32) * 3
    for d in (1, 2):
        for k in range(4):
            dx, dy, _ = orc.unit_dir(2, k)
            P = orc.roi_glcm(img, mask, 2, orc.roi_key(0, 3), 8, k, d)
            ref = _np_glcm(img, mask, 3, 8, dx * d, dy * d)
            assert np.array_equal(P.astype(np.int64), ref)
            assert np.array_equal(P, P.T)


def test_glcm_counts_bruteforce_3d(orc):
    rng = np.random.default_rng(20)
    img = rng.integers(-50, 50, size=(4, 5, 6)).astype(np.int16)
    mask = (rng.random((4, 5, 6)) < 0.8).astype(np.int32)
    seen = set()
    for k in range(13):
        dx, dy, dz = orc.unit_dir(3, k)
        assert (dx, dy, dz) != (0, 0, 0) and (-dx, -dy, -dz) not in seen
        seen.add((dx, dy, dz))
        P = orc.roi_glcm(img, mask, 3, orc.roi_key(0, 1), 6, k, 1)
        assert np.array_equal(P.astype(np.int64), _np_glcm(img, mask, 1, 6, dx, dy, dz))
    assert len(seen) == 13


def test_glcm_2d_direction_convention(orc):
    assert [orc.unit_dir(2, k)[:2] for k in range(4)] == [(1, 0), (1, -1), (0, -1), (-1, -1)]


def test_glcm_constant_image(orc):
    img = np.full((6, 7), 1234, dtype=np.uint16)
    mask = np.ones((6, 7), dtype=np.int32)
    P = orc.roi_glcm(img, mask, 2, orc.roi_key(0, 1), 16, 0, 1)
    pairs = 6 * 6  # horizontal neighbours
    assert P[0, 0] == 2 * pairs and P.sum() == 2 * pairs
    t = _single(orc, img, mask, ng=16)
    for a in (0, 45, 90, 135):
        assert t[f"GLCM_ASM_D1_A{a}"] == 1.0
        assert t[f"GLCM_JE_D1_A{a}"] == 0.0
        assert t[f"GLCM_CONTRAST_D1_A{a}"] == 0.0
        assert t[f"GLCM_IDM_D1_A{a}"] == 1.0
        assert t[f"GLCM_CORR_D1_A{a}"] == 1.0


def test_glcm_checkerboard(orc):
    gold = json.load(open(os.path.join(GOLD, "glcm_two_level.json")))
    # an odd-sized board gives equal numbers of dark-dark and light-light
    # diagonal pairs, so both diagonal directions reach p(1,1) = p(2,2) = 1/2
    y, x = np.mgrid[0:11, 0:11]
    img = (((x + y) % 2) * 1000).astype(np.uint16)
    mask = np.ones_like(img, dtype=np.int32)
    t = _single(orc, img, mask, ng=2)
    for a, key in ((0, "horizontal"), (90, "horizontal"), (45, "diagonal"), (135, "diagonal")):
        for name, val in gold[key].items():
            assert t[f"GLCM_{name}_D1_A{a}"] == pytest.approx(val, abs=1e-12), (a, name)


def test_glcm_uneven_two_level_golden(orc):
    """Hand-derived matrices with uneven marginals: DIFENTRO = 1 bit and
    CLUSHADE = +3/4 / -3/4 pin the log base and the sign of the third-order
    cluster moment, which the checkerboard cases leave at 0."""
    gold = json.load(open(os.path.join(GOLD, "glcm_uneven_two_level.json")))
    for case, spec in gold["cases"].items():
        f = orc.glcm_features(np.array(spec["P"], dtype=np.float64))
        for name, val in spec["features"].items():
            assert f[name] == pytest.approx(val, rel=1e-12, abs=1e-12), (case, name, f[name], val)
    assert gold["cases"]["offdiag"]["features"]["DIFENTRO"] == 1.0
    assert gold["cases"]["diagonal_uneven"]["features"]["CLUSHADE"] == 0.75
    assert gold["cases"]["diagonal_uneven_mirror"]["features"]["CLUSHADE"] == -0.75


def test_glcm_difentro_clushade_bruteforce(orc):
    """DIFENTRO and CLUSHADE of random symmetric matrices (Ng <= 8) against
    their definitions written out over p_{x-y} and (i + j - 2 mu)."""
    rng = np.random.default_rng(11)
    for trial in range(30):
        ng = int(rng.integers(2, 9))
        A = rng.integers(0, 6, size=(ng, ng)).astype(np.float64)
        A[rng.random((ng, ng)) < 0.4] = 0
        P = A + A.T
        if P.sum() == 0:
            continue
        p = P / P.sum()
        i = np.arange(1, ng + 1)
        mu = float((p.sum(1) * i).sum())
        shade = sum(p[a, b] * (i[a] + i[b] - 2 * mu) ** 3 for a in range(ng) for b in range(ng))
        pd = np.array([sum(p[a, b] for a in range(ng) for b in range(ng) if abs(a - b) == k) for k in range(ng)])
        difent = -sum(v * math.log(v, 2) for v in pd if v > 0)
        f = orc.glcm_features(P)
        assert f["CLUSHADE"] == pytest.approx(shade, rel=1e-10, abs=1e-12)
        assert f["DIFENTRO"] == pytest.approx(difent, rel=1e-10, abs=1e-12)


def test_glcm_feature_identities(orc):
    rng = np.random.default_rng(5)
    for trial in range(20):
        ng = int(rng.integers(2, 9))
        A = rng.integers(0, 5, size=(ng, ng)).astype(np.float64)
        A[rng.random((ng, ng)) < 0.3] = 0
        P = A + A.T
        if P.sum() == 0:
            continue
        f = orc.glcm_features(P)
        p = P / P.sum()
        px = p.sum(1)
        hx = -sum(v * math.log2(v) for v in px if v > 0)
        assert f["ACOR"] == pytest.approx((f["SUMVAR"] + f["SUMAVE"] ** 2 - f["CONTRAST"]) / 4, rel=1e-10, abs=1e-12)
        assert f["DIS"] == pytest.approx(f["DIFAVE"], rel=1e-12)
        assert f["CONTRAST"] == pytest.approx(f["DIFVAR"] + f["DIFAVE"] ** 2, rel=1e-10, abs=1e-12)
        assert f["SUMAVE"] == pytest.approx(2 * f["JAVE"], rel=1e-12)
        assert f["CLUTEND"] == pytest.approx(f["SUMVAR"], rel=1e-10, abs=1e-12)
        if f["JVAR"] > 0:
            assert f["CLUTEND"] == pytest.approx(2 * f["JVAR"] * (1 + f["CORR"]), rel=1e-10, abs=1e-12)
        assert f["ENERGY"] ** 2 == pytest.approx(f["ASM"], rel=1e-12)
        assert (f["ID"], f["IDM"], f["JE"], f["JVAR"]) == (f["HOM1"], f["HOM2"], f["ENTROPY"], f["VARIANCE"])
        # HXY1 = HXY2 = HX + HY (c10) shows through INFOMEAS1 and INFOMEAS2
        if hx > 0:
            assert f["INFOMEAS1"] == pytest.approx((f["JE"] - 2 * hx) / hx, rel=1e-10, abs=1e-12)
        assert f["INFOMEAS2"] == pytest.approx(math.sqrt(max(0.0, 1 - math.exp(-2 * (2 * hx - f["JE"])))),
                                               rel=1e-10, abs=1e-12)
        assert 0 <= f["INFOMEAS2"] < 1 and -1 - 1e-12 <= f["INFOMEAS1"] <= 1e-12
        assert 0 < f["ASM"] <= 1 and f["JMAX"] == pytest.approx(p.max())
        assert -1 - 1e-9 <= f["CORR"] <= 1 + 1e-9


def test_glcm_transpose_symmetry(orc):
    # Transposing the image swaps the 0 and 90 degree directions and maps
    # 45 degrees onto 45 degrees, 135 onto 135; the direction mean is invariant.
    rng = np.random.default_rng(6)
    img = rng.integers(0, 300, size=(12, 15)).astype(np.uint16)
    mask = np.ones_like(img, dtype=np.int32)
    a = _single(orc, img, mask, ng=8)
    b = _single(orc, np.ascontiguousarray(img.T), np.ascontiguousarray(mask.T), ng=8)
    for n in orc.GLCM_NAMES:
        assert b[f"GLCM_{n}_D1_A90"] == pytest.approx(a[f"GLCM_{n}_D1_A0"], rel=1e-12, abs=1e-12)
        assert b[f"GLCM_{n}_D1"] == pytest.approx(a[f"GLCM_{n}_D1"], rel=1e-12, abs=1e-12)


def test_glcm_no_pairs_is_nan(orc):
    img = np.array([[5, 0, 9]], dtype=np.uint16)
    mask = np.array([[1, 0, 1]], dtype=np.int32)
    t = _single(orc, img, mask, ng=4)
    assert math.isnan(t["GLCM_ASM_D1_A0"]) and math.isnan(t["GLCM_ASM_D1"])
    mask2 = np.array([[1, 1, 0]], dtype=np.int32)
    t2 = _single(orc, img, mask2, ng=4)
    # one horizontal pair (bins 3 and 0): p(1,4) = p(4,1) = 1/2
    assert t2["GLCM_ASM_D1_A0"] == 0.5 and math.isnan(t2["GLCM_ASM_D1_A90"])
    assert t2["GLCM_ASM_D1"] == 0.5  # mean over the directions that have pairs


# --------------------------------------------------------------------------
# First-order statistics

@pytest.mark.parametrize("n", [2, 7, 100, 1001])
def test_stats_uniform_ramp_closed_forms(orc, n):
    img = np.arange(n, dtype=np.uint16).reshape(1, -1)
    t = _single(orc, img, np.ones_like(img, dtype=np.int32), ng=4)
    assert t["MEAN"] == pytest.approx((n - 1) / 2, rel=1e-14)
    assert t["VARIANCE"] == pytest.approx(n * (n + 1) / 12, rel=1e-13)
    assert t["VARIANCE_BIASED"] == pytest.approx((n * n - 1) / 12, rel=1e-13)
    assert t["SKEWNESS"] == pytest.approx(0, abs=1e-12)
    assert t["KURTOSIS"] == pytest.approx(0.6 * (3 * n * n - 7) / (n * n - 1), rel=1e-12)
    assert t["HYPERSKEWNESS"] == pytest.approx(0, abs=1e-12)
    assert t["MEAN_ABSOLUTE_DEVIATION"] == pytest.approx(np.mean(np.abs(np.arange(n) - (n - 1) / 2)), rel=1e-13)
    assert t["ENERGY"] == (n - 1) * n * (2 * n - 1) / 6
    assert t["INTEGRATED_INTENSITY"] == n * (n - 1) / 2
    assert t["MODE"] == 0 and t["MODE_PROBABILITY"] == pytest.approx(1 / n)


@pytest.mark.parametrize("dtype,seed", [(np.uint16, 0), (np.int16, 1), (np.float32, 2)])
def test_stats_vs_scipy_numpy(orc, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.float32:
        vals = rng.gamma(2.0, 300.0, size=777).astype(np.float32)
    elif dtype == np.int16:
        vals = rng.integers(-1000, 3000, size=777).astype(np.int16)
    else:
        vals = rng.integers(0, 60, size=777).astype(np.uint16)
    img = vals.reshape(21, 37)
    t = _single(orc, img, np.ones_like(img, dtype=np.int32), ng=4, hist_bins=64)
    v = vals.astype(np.float64)
    m2 = scipy.stats.moment(v, 2)
    assert t["MEAN"] == pytest.approx(v.mean(), rel=1e-13)
    assert t["VARIANCE"] == pytest.approx(np.var(v, ddof=1), rel=1e-12)
    assert t["STDDEV_BIASED"] == pytest.approx(np.std(v), rel=1e-12)
    assert t["SKEWNESS"] == pytest.approx(scipy.stats.skew(v), rel=1e-10, abs=1e-12)
    assert t["KURTOSIS"] == pytest.approx(scipy.stats.kurtosis(v, fisher=False), rel=1e-10)
    assert t["EXCESS_KURTOSIS"] == pytest.approx(scipy.stats.kurtosis(v, fisher=True), rel=1e-10)
    assert t["HYPERSKEWNESS"] == pytest.approx(scipy.stats.moment(v, 5) / m2 ** 2.5, rel=1e-10, abs=1e-12)
    assert t["HYPERFLATNESS"] == pytest.approx(scipy.stats.moment(v, 6) / m2 ** 3, rel=1e-10)
    assert t["STANDARD_ERROR"] == pytest.approx(scipy.stats.sem(v), rel=1e-12)
    assert t["ROOT_MEAN_SQUARED"] == pytest.approx(np.sqrt(np.mean(v * v)), rel=1e-13)
    for q, name in ((1, "P01"), (10, "P10"), (25, "P25"), (50, "MEDIAN"), (75, "P75"), (90, "P90"), (99, "P99")):
        assert t[name] == pytest.approx(np.percentile(v, q, method="linear"), rel=1e-14, abs=1e-12)
    assert t["INTERQUARTILE_RANGE"] == pytest.approx(scipy.stats.iqr(v), rel=1e-13, abs=1e-12)
    mode = scipy.stats.mode(v, keepdims=False)
    assert t["MODE"] == mode.mode and t["MODE_PROBABILITY"] == pytest.approx(mode.count / v.size)
    counts, _ = np.histogram(v, bins=64, range=(v.min(), v.max()))
    assert t["ENTROPY"] == pytest.approx(scipy.stats.entropy(counts, base=2), rel=1e-12)
    assert t["UNIFORMITY"] == pytest.approx(np.sum((counts / v.size) ** 2), rel=1e-12)
    assert t["MEDIAN_ABSOLUTE_DEVIATION"] == pytest.approx(np.mean(np.abs(v - np.median(v))), rel=1e-12)
    p10, p90 = np.percentile(v, [10, 90])
    sel = v[(v >= p10) & (v <= p90)]
    assert t["ROBUST_MEAN"] == pytest.approx(sel.mean(), rel=1e-13)
    assert t["ROBUST_MEAN_ABSOLUTE_DEVIATION"] == pytest.approx(np.mean(np.abs(sel - sel.mean())), rel=1e-12)


def test_stats_degenerate(orc):
    img = np.array([[4242]], dtype=np.uint16)
    t = _single(orc, img, np.ones_like(img, dtype=np.int32), ng=4)
    assert t["VARIANCE"] == 0 and t["STDDEV"] == 0 and t["STANDARD_ERROR"] == 0
    assert t["SKEWNESS"] == 0 and t["KURTOSIS"] == 0 and t["HYPERFLATNESS"] == 0
    assert t["MEDIAN"] == 4242 and t["P99"] == 4242 and t["MODE_PROBABILITY"] == 1
    assert t["ENTROPY"] == 0 and t["UNIFORMITY"] == 1
    assert math.isnan(t["GLCM_ASM_D1"])
    z = np.zeros((2, 2), dtype=np.uint16)
    t = _single(orc, z, np.ones_like(z, dtype=np.int32), ng=4)
    assert math.isnan(t["INT_M10"] / 1) or True  # M10 = 0 is finite
    assert math.isnan(t["WEIGHTED_CENTROID_X"]) and math.isnan(t["INT_MU20"]) and math.isnan(t["COV"])
    assert math.isnan(t["UNIFORMITY_PIU"])


def test_weighted_centroid_and_mass_displacement(orc):
    img = np.zeros((5, 9), dtype=np.uint16)
    img[2, 1] = 10
    img[2, 7] = 30
    mask = (img > 0).astype(np.int32)
    t = _single(orc, img, mask, ng=4)
    assert t["WEIGHTED_CENTROID_X"] == pytest.approx((1 * 10 + 7 * 30) / 40)
    assert t["CENTROID_X"] == 4.0 and t["WEIGHTED_CENTROID_Y"] == 2.0
    assert t["MASS_DISPLACEMENT"] == pytest.approx(5.5 - 4.0)


# --------------------------------------------------------------------------
# Moments

@pytest.mark.parametrize("w,h", [(1, 1), (3, 5), (8, 2), (11, 7)])
def test_rectangle_central_moments(orc, w, h):
    img = np.full((h + 4, w + 6), 9, dtype=np.uint16)
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[2:2 + h, 3:3 + w] = 1
    t = _single(orc, img, mask, ng=4)
    for pre, scale in (("BIN", 1.0), ("INT", 9.0)):
        assert t[f"{pre}_M00"] == scale * w * h
        assert t[f"{pre}_MU20"] == pytest.approx(scale * h * w * (w * w - 1) / 12, rel=1e-13, abs=1e-12)
        assert t[f"{pre}_MU02"] == pytest.approx(scale * w * h * (h * h - 1) / 12, rel=1e-13, abs=1e-12)
        for nm in ("MU11", "MU30", "MU03", "MU21", "MU12", "MU10", "MU01"):
            assert t[f"{pre}_{nm}"] == pytest.approx(0, abs=1e-9)
        # raw moments of the rectangle in bbox-local coordinates
        assert t[f"{pre}_M10"] == pytest.approx(scale * h * w * (w - 1) / 2)
        assert t[f"{pre}_M21"] == pytest.approx(scale * (w - 1) * w * (2 * w - 1) / 6 * (h - 1) * h / 2)
    # constant weighting c: mu_pq and M_pq scale by c, so eta_pq and nu_pq
    # scale by c^(-(p+q)/2); Hu1 (order 2) by 1/c, Hu2 by 1/c^2
    for nm, k in (("ETA20", 1), ("ETA02", 1), ("NU11", 1), ("NU21", 1.5), ("HU1", 1), ("HU2", 2)):
        assert t[f"INT_{nm}"] == pytest.approx(t[f"BIN_{nm}"] * 9.0 ** -k, rel=1e-12, abs=1e-15)


def _disc(r, pad=3):
    n = 2 * r + 1 + 2 * pad
    y, x = np.mgrid[0:n, 0:n]
    c = r + pad
    return ((x - c) ** 2 + (y - c) ** 2 <= r * r).astype(np.int32)


def test_disc_hu1_limit(orc):
    prev = None
    for r in (10, 40, 120):
        m = _disc(r)
        t = _single(orc, m.astype(np.uint16), m, ng=0 or 2)
        err = abs(t["BIN_HU1"] - 1 / (2 * math.pi))
        assert err < 2e-3 * 40 / r
        assert t["BIN_HU2"] < 1e-6 and abs(t["BIN_ETA11"]) < 1e-12
        if prev is not None:
            assert err < prev
        prev = err


def test_hu_invariance_translation_rotation_and_flip(orc):
    rng = np.random.default_rng(7)
    img = np.zeros((40, 50), dtype=np.float32)
    mask = np.zeros((40, 50), dtype=np.int32)
    yy, xx = np.mgrid[0:40, 0:50]
    # axis-aligned ellipse plus a bump at 30 degrees: no mirror symmetry
    blob = (((xx - 17) / 9.0) ** 2 + ((yy - 15) / 5.0) ** 2 <= 1) | \
        ((xx - 17 - 8 * math.cos(0.5236)) ** 2 + (yy - 15 - 8 * math.sin(0.5236)) ** 2 <= 9)
    mask[blob] = 1
    img[blob] = rng.uniform(0.5, 2.0, size=blob.sum())
    base = _single(orc, img, mask, ng=4)
    variants = {
        "shift": (np.roll(np.roll(img, 5, 0), 11, 1), np.roll(np.roll(mask, 5, 0), 11, 1)),
        "rot90": (np.rot90(img).copy(), np.rot90(mask).copy()),
        "rot180": (np.rot90(img, 2).copy(), np.rot90(mask, 2).copy()),
    }
    for k, (im, ma) in variants.items():
        t = _single(orc, im, ma, ng=4)
        for pre in ("INT", "BIN"):
            for h in range(1, 8):
                a, b = t[f"{pre}_HU{h}"], base[f"{pre}_HU{h}"]
                assert a == pytest.approx(b, rel=1e-9, abs=0), (k, pre, h)
    t = _single(orc, np.fliplr(img).copy(), np.fliplr(mask).copy(), ng=4)
    for pre in ("INT", "BIN"):
        for h in range(1, 7):
            assert t[f"{pre}_HU{h}"] == pytest.approx(base[f"{pre}_HU{h}"], rel=1e-9, abs=0)
        assert t[f"{pre}_HU7"] == pytest.approx(-base[f"{pre}_HU7"], rel=1e-9, abs=0)
        assert abs(base[f"{pre}_HU7"]) > 1e-12


def test_moments_vs_bruteforce_numpy(orc):
    rng = np.random.default_rng(8)
    img = rng.integers(0, 1000, size=(9, 11)).astype(np.uint16)
    mask = (rng.random((9, 11)) < 0.6).astype(np.int32)
    t = _single(orc, img, mask, ng=4)
    ys, xs = np.nonzero(mask)
    w = img[ys, xs].astype(np.float64)
    x = xs - xs.min()
    y = ys - ys.min()
    xb, yb = (x * w).sum() / w.sum(), (y * w).sum() / w.sum()
    for p in range(4):
        for q in range(4 - p):
            assert t[f"INT_M{p}{q}"] == pytest.approx(np.sum(x ** p * y ** q * w), rel=1e-13)
            mu = np.sum((x - xb) ** p * (y - yb) ** q * w)
            assert t[f"INT_MU{p}{q}"] == pytest.approx(mu, rel=1e-9, abs=1e-6)
            assert t[f"INT_NU{p}{q}"] == pytest.approx(np.sum(x ** p * y ** q * w) / w.sum() ** (1 + (p + q) / 2),
                                                       rel=1e-12)
            if p + q >= 2:
                assert t[f"INT_ETA{p}{q}"] == pytest.approx(mu / w.sum() ** (1 + (p + q) / 2), rel=1e-9, abs=1e-12)


def test_3d_box_moments(orc):
    w, h, d = 4, 3, 5
    img = np.full((d + 2, h + 2, w + 2), 3, dtype=np.int16)
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[1:1 + d, 1:1 + h, 1:1 + w] = 2
    t = _single(orc, img, mask, ndim=3, ng=4)
    assert t["BIN_M000"] == w * h * d
    assert t["BIN_MU200"] == pytest.approx(h * d * w * (w * w - 1) / 12)
    assert t["BIN_MU020"] == pytest.approx(w * d * h * (h * h - 1) / 12)
    assert t["BIN_MU002"] == pytest.approx(w * h * d * (d * d - 1) / 12)
    for nm in ("MU110", "MU101", "MU011", "MU300", "MU111", "MU012"):
        assert t[f"BIN_{nm}"] == pytest.approx(0, abs=1e-9)
    assert t["INT_ETA200"] == pytest.approx(t["BIN_MU200"] * 3 / (3 * w * h * d) ** (1 + 2 / 3), rel=1e-12)
    # the 3D table carries no Hu or normalised raw columns (Table S5 rows 368, 370)
    assert "INT_HU1" not in t and "BIN_NU000" not in t


# --------------------------------------------------------------------------
# Gradient oracle vs central finite differences (FP64, h = 1e-3)

SMOOTH = ["MEAN", "VARIANCE", "VARIANCE_BIASED", "STDDEV", "STDDEV_BIASED", "SKEWNESS", "KURTOSIS",
          "EXCESS_KURTOSIS", "HYPERSKEWNESS", "HYPERFLATNESS", "ENERGY", "ROOT_MEAN_SQUARED", "STANDARD_ERROR",
          "MEAN_ABSOLUTE_DEVIATION", "INTEGRATED_INTENSITY", "WEIGHTED_CENTROID_X", "WEIGHTED_CENTROID_Y",
          "MASS_DISPLACEMENT", "COV", "EDGE_INTEGRATED_INTENSITY", "EDGE_MEAN_INTENSITY", "EDGE_STDDEV_INTENSITY"]


def _moment_names(ndim):
    out = []
    if ndim == 2:
        for p in range(4):
            for q in range(4 - p):
                out += [f"INT_M{p}{q}", f"INT_NU{p}{q}"]
                if p + q != 1:  # first-order central moments are identically 0
                    out.append(f"INT_MU{p}{q}")
                if p + q >= 2:
                    out.append(f"INT_ETA{p}{q}")
        out += [f"INT_HU{h}" for h in range(1, 8)]
    else:
        for p in range(4):
            for q in range(4 - p):
                for r in range(4 - p - q):
                    out.append(f"INT_M{p}{q}{r}")
                    if p + q + r != 1:
                        out.append(f"INT_MU{p}{q}{r}")
                    if p + q + r >= 2:
                        out.append(f"INT_ETA{p}{q}{r}")
        out.append("WEIGHTED_CENTROID_Z")
    return out


@pytest.mark.parametrize("ndim", [2, 3])
def test_gradient_vs_finite_differences(orc, ndim):
    rng = np.random.default_rng(30 + ndim)
    shape = (7, 9) if ndim == 2 else (3, 4, 5)
    img = rng.uniform(50, 150, size=shape)
    mask = rng.integers(1, 3, size=shape).astype(np.int32)
    mask.flat[0] = 0
    names = SMOOTH + _moment_names(ndim)
    t = orc.extract(img, mask, ndim, ng=0)
    nroi = len(t["LABEL"])
    gtab = {}
    for nm in names:
        scale = np.abs(t[nm]) + 1e-3
        gtab[nm] = rng.normal(size=nroi) / scale
    g = orc.grad(img, mask, ndim, gtab)

    def loss(im):
        tt = orc.extract(im, mask, ndim, ng=0)
        return sum(float(np.sum(gtab[nm] * tt[nm])) for nm in names)

    h = 1e-3
    flat = np.flatnonzero(mask.ravel() > 0)
    for idx in rng.choice(flat, size=12, replace=False):
        ip = img.copy()
        im = img.copy()
        ip.flat[idx] += h
        im.flat[idx] -= h
        fd = (loss(ip) - loss(im)) / (2 * h)
        assert g.flat[idx] == pytest.approx(fd, rel=1e-5, abs=1e-7), idx
    assert np.all(g.ravel()[mask.ravel() == 0] == 0)


def test_gradient_single_feature_closed_forms(orc):
    rng = np.random.default_rng(40)
    img = rng.uniform(10, 20, size=(4, 6))
    mask = np.ones((4, 6), dtype=np.int32)
    N = img.size
    g = orc.grad(img, mask, 2, {"MEAN": np.array([1.0])})
    assert np.allclose(g, 1.0 / N, rtol=1e-14)
    g = orc.grad(img, mask, 2, {"VARIANCE": np.array([1.0])})
    assert np.allclose(g, 2 * (img - img.mean()) / (N - 1), rtol=1e-12)
    g = orc.grad(img, mask, 2, {"INT_M11": np.array([1.0])})
    y, x = np.mgrid[0:4, 0:6]
    assert np.allclose(g, x * y, rtol=1e-14)


def test_small_closed_forms_dispersion(orc):
    # ROI values {1, 3} inside an image whose range is [0, 10] (hand-computed):
    # mean 2, unbiased var 2, COV = sqrt(2)/2, PIU = 100 (1 - 2/4) = 50,
    # covered range = 2/10, P25 = 1.5, P75 = 2.5, QCOD = 1/4, MAD = 1
    img = np.array([[1, 3, 0, 10]], dtype=np.uint16)
    mask = np.array([[1, 1, 0, 0]], dtype=np.int32)
    t = _single(orc, img, mask, ng=2)
    assert t["COV"] == pytest.approx(math.sqrt(2) / 2, rel=1e-15)
    assert t["UNIFORMITY_PIU"] == pytest.approx(50.0, rel=1e-15)
    assert t["COVERED_IMAGE_INTENSITY_RANGE"] == pytest.approx(0.2, rel=1e-15)
    assert (t["P25"], t["P75"], t["QCOD"]) == (1.5, 2.5, 0.25)
    assert t["MEAN_ABSOLUTE_DEVIATION"] == 1.0 and t["RANGE"] == 2.0
    assert t["ROBUST_MEAN"] != t["ROBUST_MEAN"]  # no value inside [P10, P90] = [1.2, 2.8]: NaN


# --------------------------------------------------------------------------
# Edge intensity statistics (Table S1 rows 3-7, Table S5): edge pixels are
# the ROI pixels a face-connected erosion removes (scipy.ndimage, with the
# image border counted as outside), statistics by NumPy over them.

def _edge_ref(img, mask, label):
    import scipy.ndimage as ndi

    m = mask == label
    cross = ndi.generate_binary_structure(m.ndim, 1)
    inner = ndi.binary_erosion(m, structure=cross, border_value=0)
    v = img[m & ~inner].astype(np.float64)
    return {"EDGE_INTEGRATED_INTENSITY": v.sum(), "EDGE_MAX_INTENSITY": v.max(), "EDGE_MIN_INTENSITY": v.min(),
            "EDGE_MEAN_INTENSITY": v.mean(), "EDGE_STDDEV_INTENSITY": v.std(ddof=1) if v.size > 1 else 0.0}, v.size


def test_edge_rectangle_ring(orc):
    """A 3 x 4 rectangle inside the image: 10 ring pixels, 2 interior ones."""
    img = np.arange(1, 8 * 9 + 1, dtype=np.uint16).reshape(8, 9) * 7
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[2:5, 3:7] = 4
    t = _single(orc, img, mask, ng=4)
    ring = np.concatenate([img[2, 3:7], img[4, 3:7], img[3, [3, 6]]]).astype(np.float64)
    assert ring.size == 10
    assert t["EDGE_INTEGRATED_INTENSITY"] == ring.sum()
    assert t["EDGE_MIN_INTENSITY"] == ring.min() and t["EDGE_MAX_INTENSITY"] == ring.max()
    assert t["EDGE_MEAN_INTENSITY"] == pytest.approx(ring.mean(), rel=1e-15)
    assert t["EDGE_STDDEV_INTENSITY"] == pytest.approx(ring.std(ddof=1), rel=1e-14)


def test_edge_single_pixel_and_line(orc):
    img = np.full((5, 6), 9, dtype=np.uint16)
    img[1, 1] = 321
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[1, 1] = 1          # one pixel: its own edge, deviation 0
    mask[3, 0:6] = 2        # full-width line: every pixel is an edge pixel
    img[3, :] = [5, 1, 4, 1, 5, 9]
    t = orc.extract(img, mask, 2, ng=4)
    assert t["EDGE_INTEGRATED_INTENSITY"][0] == 321 and t["EDGE_STDDEV_INTENSITY"][0] == 0
    assert t["EDGE_INTEGRATED_INTENSITY"][1] == 25 and t["EDGE_MEAN_INTENSITY"][1] == pytest.approx(25 / 6)
    assert t["EDGE_STDDEV_INTENSITY"][1] == pytest.approx(np.std([5, 1, 4, 1, 5, 9], ddof=1), rel=1e-14)


def test_edge_cube_3d_face_neighbours(orc):
    """3 x 3 x 3 cube: with face neighbours only the centre voxel is inner."""
    img = np.random.default_rng(7).integers(-500, 500, size=(5, 5, 5)).astype(np.int16)
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[1:4, 1:4, 1:4] = 3
    t = _single(orc, img, mask, ndim=3, ng=4)
    ref, n = _edge_ref(img, mask, 3)
    assert n == 26
    sel = np.ones((3, 3, 3), bool)
    sel[1, 1, 1] = False
    assert ref["EDGE_INTEGRATED_INTENSITY"] == img[1:4, 1:4, 1:4][sel].astype(np.float64).sum()
    for k, v in ref.items():
        assert t[k] == pytest.approx(v, rel=1e-13)


@pytest.mark.parametrize("ndim,seed", [(2, 1), (2, 2), (3, 3)])
def test_edge_touching_rois_and_border_vs_erosion(orc, ndim, seed):
    """Random touching blobs, some cut by the image border: a pixel next to
    another label or to the border is an edge pixel."""
    rng = np.random.default_rng(seed)
    shape = (24, 29) if ndim == 2 else (9, 12, 13)
    img = rng.gamma(2.0, 300.0, size=shape).astype(np.float32)
    mask = np.zeros(shape, dtype=np.int32)
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    for lab in range(1, 7):
        c = [rng.uniform(-2, s + 2) for s in shape]
        r = rng.uniform(2.5, 6.0)
        d2 = sum((g - ci) ** 2 for g, ci in zip(grids, c))
        mask[d2 <= r * r] = lab
    t = orc.extract(img, mask, ndim, ng=4)
    for row, lab in enumerate(t["LABEL"].astype(int)):
        ref, _ = _edge_ref(img, mask, lab)
        for k, v in ref.items():
            assert t[k][row] == pytest.approx(v, rel=1e-12, abs=1e-9), (lab, k)


def test_gradient_edge_features_closed_forms(orc):
    """Edge mean and integrated intensity: constant gradient on the edge
    ring, zero inside; edge deviation: (I - mean_E) / ((n_E - 1) std_E)."""
    rng = np.random.default_rng(41)
    img = rng.uniform(10, 20, size=(6, 7))
    mask = np.zeros((6, 7), dtype=np.int32)
    mask[1:5, 1:6] = 1
    ring = mask.astype(bool).copy()
    ring[2:4, 2:5] = False
    ne = ring.sum()
    g = orc.grad(img, mask, 2, {"EDGE_MEAN_INTENSITY": np.array([1.0])})
    assert np.allclose(g[ring], 1.0 / ne, rtol=1e-14) and np.all(g[~ring] == 0)
    g = orc.grad(img, mask, 2, {"EDGE_INTEGRATED_INTENSITY": np.array([2.5])})
    assert np.allclose(g[ring], 2.5, rtol=1e-14) and np.all(g[~ring] == 0)
    v = img[ring]
    g = orc.grad(img, mask, 2, {"EDGE_STDDEV_INTENSITY": np.array([1.0])})
    assert np.allclose(g[ring], (v - v.mean()) / ((ne - 1) * v.std(ddof=1)), rtol=1e-12)
    assert np.all(g[~ring] == 0)


# --------------------------------------------------------------------------
# NGTDM (Table S3 rows 246-250): an independent NumPy construction of the
# neighbourhood means (scipy.ndimage correlation with the 8- / 26-neighbour
# kernel) and of the five features with explicit pair arrays.

def _ngtdm_ref(img, mask, label, ng):
    import scipy.ndimage as ndi

    m = mask == label
    v = img[m].astype(np.int64)
    mn, mx = v.min(), v.max()
    lev = np.zeros(img.shape, dtype=np.int64)
    if mx > mn:
        lev[m] = np.minimum(ng * (img[m].astype(np.int64) - mn) // (mx - mn), ng - 1) + 1
    else:
        lev[m] = 1
    k = np.ones((3,) * img.ndim)
    k[(1,) * img.ndim] = 0
    s_nb = ndi.correlate(lev.astype(np.float64), k, mode="constant", cval=0.0)
    c_nb = ndi.correlate(m.astype(np.float64), k, mode="constant", cval=0.0)
    valid = m & (c_nb > 0)
    if not valid.any():
        return [np.nan] * 5
    L = lev[valid]
    A = s_nb[valid] / c_nb[valid]
    n = np.bincount(L, minlength=ng + 1)[1:].astype(np.float64)
    s = np.bincount(L, weights=np.abs(L - A), minlength=ng + 1)[1:]
    N = n.sum()
    z = n > 0
    p, sz, li = n[z] / N, s[z], np.arange(1, ng + 1, dtype=np.float64)[z]
    G = z.sum()
    ps = np.sum(p * sz)
    dl = li[:, None] - li[None, :]
    coarse = 1.0 / ps if ps > 0 else np.nan
    contrast = np.sum(p[:, None] * p[None, :] * dl ** 2) / (G * (G - 1)) * s.sum() / N if G > 1 else 0.0
    den = np.sum(np.abs((li * p)[:, None] - (li * p)[None, :]))
    busy = ps / den if den > 0 else 0.0
    cplx = np.sum(np.abs(dl) * ((p * sz)[:, None] + (p * sz)[None, :]) / (p[:, None] + p[None, :])) / N
    strength = np.sum((p[:, None] + p[None, :]) * dl ** 2) / s.sum() if s.sum() > 0 else 0.0
    return [coarse, contrast, busy, cplx, strength]


NGTDM_COLS = ["NGTDM_COARSENESS", "NGTDM_CONTRAST", "NGTDM_BUSYNESS", "NGTDM_COMPLEXITY", "NGTDM_STRENGTH"]


@pytest.mark.parametrize("ndim,seed,ng", [(2, 1, 8), (2, 2, 32), (3, 3, 16)])
def test_ngtdm_vs_numpy_construction(orc, ndim, seed, ng):
    rng = np.random.default_rng(50 + seed)
    shape = (30, 33) if ndim == 2 else (10, 12, 13)
    img = rng.integers(0, 4000, size=shape).astype(np.uint16)
    mask = np.zeros(shape, dtype=np.int32)
    grids = np.meshgrid(*[np.arange(sh) for sh in shape], indexing="ij")
    for lab in range(1, 6):  # touching blobs, some cut by the border
        c = [rng.uniform(-1, sh + 1) for sh in shape]
        r = rng.uniform(2.5, 7.0)
        mask[sum((g - ci) ** 2 for g, ci in zip(grids, c)) <= r * r] = lab
    t = orc.extract(img, mask, ndim, ng=ng)
    for row, lab in enumerate(t["LABEL"].astype(int)):
        ref = _ngtdm_ref(img, mask, lab, ng)
        for name, v in zip(NGTDM_COLS, ref):
            if np.isnan(v):
                assert np.isnan(t[name][row]), (lab, name)
            else:
                assert t[name][row] == pytest.approx(v, rel=1e-12, abs=1e-12), (lab, name)


def test_ngtdm_degenerate_cases(orc):
    img = np.full((6, 7), 100, dtype=np.uint16)
    img[0, 0] = 7
    mask = np.zeros((6, 7), dtype=np.int32)
    mask[0, 0] = 1           # single pixel: no neighbour, every NGTDM feature NaN
    mask[2:5, 2:6] = 2       # constant ROI: one grey level, no difference
    t = orc.extract(img, mask, 2, ng=8)
    assert all(np.isnan(t[c][0]) for c in NGTDM_COLS)
    assert np.isnan(t["NGTDM_COARSENESS"][1])
    assert t["NGTDM_CONTRAST"][1] == 0 and t["NGTDM_BUSYNESS"][1] == 0
    assert t["NGTDM_COMPLEXITY"][1] == 0 and t["NGTDM_STRENGTH"][1] == 0


def test_ngtdm_two_level_stripes_closed_form(orc):
    """Vertical stripes of width 1 alternating levels 1 and 2 in a 4 x 6 ROI
    filling the image (Ng = 2, min 0, max 1): every pixel is valid, and an
    interior pixel sees 6 neighbours of the other level and 2 of its own, so
    |L - A| = 3/4 there.  Checked against the NumPy construction."""
    img = np.tile(np.array([0, 1], dtype=np.uint16), (4, 3))
    mask = np.ones(img.shape, dtype=np.int32)
    t = _single(orc, img, mask, ng=2)
    ref = _ngtdm_ref(img, mask, 1, 2)
    for name, v in zip(NGTDM_COLS, ref):
        assert t[name] == pytest.approx(v, rel=1e-13)
    assert t["NGTDM_CONTRAST"] > 0 and t["NGTDM_BUSYNESS"] > 0


# --------------------------------------------------------------------------
# GLDM (Table S3 rows 251-264): the dependence matrix built independently
# with one scipy.ndimage correlation per grey level (same-level neighbour
# counts), the fourteen features from the explicit matrix, and a constant
# square whose matrix is known by hand.

GLDM_COLS = ["GLDM_" + n for n in ("SDE", "LDE", "GLN", "DN", "DNN", "GLV", "DV", "DE", "LGLE", "HGLE", "SDLGLE",
                                   "SDHGLE", "LDLGLE", "LDHGLE")]


def _gldm_matrix(img, mask, label, ng):
    import scipy.ndimage as ndi

    m = mask == label
    v = img[m].astype(np.int64)
    mn, mx = v.min(), v.max()
    lev = np.zeros(img.shape, dtype=np.int64)
    if mx > mn:
        lev[m] = np.minimum(ng * (img[m].astype(np.int64) - mn) // (mx - mn), ng - 1) + 1
    else:
        lev[m] = 1
    k = np.ones((3,) * img.ndim)
    k[(1,) * img.ndim] = 0
    nj = 3 ** img.ndim
    P = np.zeros((ng, nj))
    for i in range(1, ng + 1):
        ind = (lev == i) & m
        if not ind.any():
            continue
        same = ndi.correlate(ind.astype(np.int64), k.astype(np.int64), mode="constant", cval=0)
        P[i - 1] = np.bincount(same[ind] + 1, minlength=nj + 1)[1:]
    return P


def _gldm_features(P):
    N = P.sum()
    i = np.arange(1, P.shape[0] + 1, dtype=np.float64)[:, None]
    j = np.arange(1, P.shape[1] + 1, dtype=np.float64)[None, :]
    p = P / N
    mui, muj = np.sum(p * i), np.sum(p * j)
    nz = p > 0
    return [np.sum(P / j ** 2) / N, np.sum(P * j ** 2) / N, np.sum(P.sum(1) ** 2) / N, np.sum(P.sum(0) ** 2) / N,
            np.sum(P.sum(0) ** 2) / N ** 2, np.sum(p * (i - mui) ** 2), np.sum(p * (j - muj) ** 2),
            -np.sum(p[nz] * np.log2(p[nz])), np.sum(P / i ** 2) / N, np.sum(P * i ** 2) / N,
            np.sum(P / (i ** 2 * j ** 2)) / N, np.sum(P * i ** 2 / j ** 2) / N, np.sum(P * j ** 2 / i ** 2) / N,
            np.sum(P * i ** 2 * j ** 2) / N]


@pytest.mark.parametrize("ndim,seed,ng", [(2, 1, 8), (2, 2, 32), (3, 3, 16)])
def test_gldm_vs_numpy_construction(orc, ndim, seed, ng):
    rng = np.random.default_rng(70 + seed)
    shape = (30, 33) if ndim == 2 else (10, 12, 13)
    # few distinct values so that same-level neighbours are common
    img = (rng.integers(0, 6, size=shape) * 700).astype(np.uint16)
    mask = np.zeros(shape, dtype=np.int32)
    grids = np.meshgrid(*[np.arange(sh) for sh in shape], indexing="ij")
    for lab in range(1, 6):  # touching blobs, some cut by the border
        c = [rng.uniform(-1, sh + 1) for sh in shape]
        r = rng.uniform(2.5, 7.0)
        mask[sum((g - ci) ** 2 for g, ci in zip(grids, c)) <= r * r] = lab
    t = orc.extract(img, mask, ndim, ng=ng)
    for row, lab in enumerate(t["LABEL"].astype(int)):
        P = _gldm_matrix(img, mask, lab, ng)
        assert P.sum() == np.count_nonzero(mask == lab)
        for name, v in zip(GLDM_COLS, _gldm_features(P)):
            assert t[name][row] == pytest.approx(v, rel=1e-12, abs=1e-12), (lab, name)


def test_gldm_constant_square_closed_form(orc):
    """A constant 3 x 3 ROI in 2D: one grey level; 4 corners with 3
    neighbours (dependence 4), 4 edge centres with 5 (dependence 6), the
    centre with 8 (dependence 9), so P(1, 4) = P(1, 6) = 4, P(1, 9) = 1."""
    img = np.full((5, 5), 300, dtype=np.uint16)
    mask = np.zeros((5, 5), dtype=np.int32)
    mask[1:4, 1:4] = 1
    t = _single(orc, img, mask, ng=16)
    n, deps = 9.0, {4: 4.0, 6: 4.0, 9: 1.0}
    sde = sum(c / d ** 2 for d, c in deps.items()) / n
    lde = sum(c * d ** 2 for d, c in deps.items()) / n
    muj = sum(c * d for d, c in deps.items()) / n
    want = {"SDE": sde, "LDE": lde, "GLN": n, "DN": 33.0 / n, "DNN": 33.0 / n ** 2, "GLV": 0.0,
            "DV": sum(c * (d - muj) ** 2 for d, c in deps.items()) / n,
            "DE": -sum((c / n) * np.log2(c / n) for c in deps.values()), "LGLE": 1.0, "HGLE": 1.0,
            "SDLGLE": sde, "SDHGLE": sde, "LDLGLE": lde, "LDHGLE": lde}
    for k, v in want.items():
        assert t["GLDM_" + k] == pytest.approx(v, rel=1e-14, abs=1e-15), k
    assert lde == pytest.approx(289.0 / 9.0)


def test_gldm_checkerboard_and_isolated_pixels(orc):
    """A two-level checkerboard: in 2D every same-level neighbour is
    diagonal, so each of the 36 interior pixels has dependence 5.  Isolated
    pixels have dependence 1 at any level: SDE = LDE = 1, DN = N, DNN = 1,
    DV = 0."""
    yy, xx = np.mgrid[0:8, 0:8]
    img = ((xx + yy) % 2).astype(np.uint16)
    mask = np.ones((8, 8), dtype=np.int32)
    t = _single(orc, img, mask, ng=2)
    P = _gldm_matrix(img, mask, 1, 2)
    assert P[:, 4].sum() == 36  # the 6 x 6 interior
    for name, v in zip(GLDM_COLS, _gldm_features(P)):
        assert t[name] == pytest.approx(v, rel=1e-13), name
    mask = np.zeros((9, 9), dtype=np.int32)
    mask[::3, ::3] = 1       # 9 pixels, no two adjacent
    img = (np.arange(81).reshape(9, 9) * 5).astype(np.uint16)
    t = _single(orc, img, mask, ng=4)
    assert t["GLDM_SDE"] == 1.0 and t["GLDM_LDE"] == 1.0
    assert t["GLDM_DN"] == 9.0 and t["GLDM_DNN"] == 1.0 and t["GLDM_DV"] == 0.0


# --------------------------------------------------------------------------
# GLRLM and GLSZM (optional families of the oracle).  Runs along a direction
# v are the connected components of one level's indicator under a structure
# holding only the centre and +-v; zones are its components under the full
# 3^n structure (scipy.ndimage.label).  The features follow from the item
# lists with np.unique.

RL_COLS = ["GLRLM_" + n for n in ("SRE", "LRE", "GLNU", "GLNUN", "RLNU", "RLNUN", "RP", "GLV", "RV", "RE", "LGLRE",
                                  "HGLRE", "SRLGLE", "SRHGLE", "LRLGLE", "LRHGLE")]
SZ_COLS = ["GLSZM_" + n for n in ("SAE", "LAE", "GLNU", "GLNUN", "SZNU", "SZNUN", "ZP", "GLV", "ZV", "ZE", "LGLZE",
                                  "HGLZE", "SALGLE", "SAHGLE", "LALGLE", "LAHGLE", "GLM", "ZSM")]


def _levels(img, mask, label, ng):
    m = mask == label
    v = img[m].astype(np.int64)
    mn, mx = v.min(), v.max()
    lev = np.zeros(img.shape, dtype=np.int64)
    lev[m] = np.minimum(ng * (v - mn) // (mx - mn), ng - 1) + 1 if mx > mn else 1
    return lev


def _axes(ndim):
    """One vector of each of the 4 (2D) / 13 (3D) lattice axes."""
    out = []
    for v in np.ndindex(*(3,) * ndim):
        v = np.array(v) - 1
        nz = np.flatnonzero(v)
        if nz.size and v[nz[0]] > 0:
            out.append(v)
    return out


def _components(lev, structure):
    import scipy.ndimage as ndi

    lv, sz = [], []
    for L in np.unique(lev[lev > 0]):
        lab, n = ndi.label(lev == L, structure=structure)
        counts = np.bincount(lab.ravel())[1:]
        lv += [L] * n
        sz += counts.tolist()
    return np.array(lv, dtype=np.float64), np.array(sz, dtype=np.float64)


def _item_features(i, s, npix):
    M = i.size
    _, ni = np.unique(i, return_counts=True)
    _, ns = np.unique(s, return_counts=True)
    _, nc = np.unique(np.stack([i, s]), axis=1, return_counts=True)
    pc = nc / M
    return [np.mean(1 / s ** 2), np.mean(s ** 2), np.sum(ni ** 2) / M, np.sum(ni ** 2) / M ** 2,
            np.sum(ns ** 2) / M, np.sum(ns ** 2) / M ** 2, M / npix, np.var(i), np.var(s),
            -np.sum(pc * np.log2(pc)), np.mean(1 / i ** 2), np.mean(i ** 2), np.mean(1 / (i * s) ** 2),
            np.mean(i ** 2 / s ** 2), np.mean(s ** 2 / i ** 2), np.mean((i * s) ** 2), np.mean(i), np.mean(s)]


def _glrlm_ref(lev, npix):
    acc = np.zeros(16)
    axes = _axes(lev.ndim)
    for v in axes:
        st = np.zeros((3,) * lev.ndim, dtype=bool)
        c = np.ones(lev.ndim, dtype=int)
        st[tuple(c)] = st[tuple(c + v)] = st[tuple(c - v)] = True
        i, s = _components(lev, st)
        acc += np.array(_item_features(i, s, npix)[:16])
    return acc / len(axes)


def _glszm_ref(lev, npix):
    i, s = _components(lev, np.ones((3,) * lev.ndim, dtype=bool))
    return _item_features(i, s, npix)


@pytest.mark.parametrize("ndim,seed,ng", [(2, 1, 4), (2, 2, 32), (3, 3, 3), (3, 4, 16)])
def test_glrlm_glszm_vs_ndimage_construction(orc, ndim, seed, ng):
    rng = np.random.default_rng(90 + seed)
    shape = (26, 29) if ndim == 2 else (9, 11, 12)
    img = (rng.integers(0, 4, size=shape) * 900 + rng.integers(0, 2, size=shape)).astype(np.uint16)
    mask = np.zeros(shape, dtype=np.int32)
    grids = np.meshgrid(*[np.arange(sh) for sh in shape], indexing="ij")
    for lab in range(1, 5):  # touching blobs, some cut by the border
        c = [rng.uniform(-1, sh + 1) for sh in shape]
        r = rng.uniform(2.5, 7.0)
        mask[sum((g - ci) ** 2 for g, ci in zip(grids, c)) <= r * r] = lab
    t = orc.extract(img, mask, ndim, ng=ng, families=("glrlm", "glszm"))
    for row, lab in enumerate(t["LABEL"].astype(int)):
        lev = _levels(img, mask, lab, ng)
        npix = np.count_nonzero(mask == lab)
        for name, v in zip(RL_COLS, _glrlm_ref(lev, npix)):
            assert t[name][row] == pytest.approx(v, rel=1e-12, abs=1e-12), (lab, name)
        for name, v in zip(SZ_COLS, _glszm_ref(lev, npix)):
            assert t[name][row] == pytest.approx(v, rel=1e-12, abs=1e-12), (lab, name)


def test_glrlm_line_closed_form(orc):
    """A constant horizontal line of L pixels: one run of length L along 0
    degrees, L runs of length 1 along 45, 90 and 135 degrees; each feature is
    the mean of the four directions (each direction has one level and one
    run length, so both normalised non-uniformities are 1)."""
    L = 7
    img = np.full((3, 10), 50, dtype=np.uint16)
    mask = np.zeros((3, 10), dtype=np.int32)
    mask[1, 2:2 + L] = 1
    t = _single(orc, img, mask, ng=8, families=("glrlm",))
    want = {"SRE": (1 / L ** 2 + 3) / 4, "LRE": (L ** 2 + 3) / 4, "GLNU": (1 + 3 * L) / 4,
            "GLNUN": 1.0, "RLNU": (1 + 3 * L) / 4, "RLNUN": 1.0, "RP": (1 / L + 3) / 4,
            "GLV": 0.0, "RV": 0.0, "RE": 0.0, "LGLRE": 1.0, "HGLRE": 1.0, "SRLGLE": (1 / L ** 2 + 3) / 4,
            "SRHGLE": (1 / L ** 2 + 3) / 4, "LRLGLE": (L ** 2 + 3) / 4, "LRHGLE": (L ** 2 + 3) / 4}
    for k, v in want.items():
        assert t["GLRLM_" + k] == pytest.approx(v, rel=1e-14, abs=1e-15), k
    assert not any(k.startswith("GLSZM_") for k in t)


def test_glszm_checkerboard_is_two_zones(orc):
    """A two-level checkerboard: with 8-connectivity the diagonal neighbours
    join every cell of one colour into a single zone (with 4-connectivity
    each cell would be its own zone)."""
    n = 6
    yy, xx = np.mgrid[0:n, 0:n]
    img = ((xx + yy) % 2).astype(np.uint16)
    mask = np.ones((n, n), dtype=np.int32)
    t = _single(orc, img, mask, ng=2, families=("glszm",))
    s = n * n / 2
    want = {"ZP": 2 / n ** 2, "SAE": 1 / s ** 2, "LAE": s ** 2, "GLNU": 1.0, "GLNUN": 0.5, "SZNU": 2.0,
            "SZNUN": 1.0, "ZE": 1.0, "GLV": 0.25, "ZV": 0.0, "GLM": 1.5, "ZSM": s,
            "LGLZE": (1 + 1 / 4) / 2, "HGLZE": (1 + 4) / 2}
    for k, v in want.items():
        assert t["GLSZM_" + k] == pytest.approx(v, rel=1e-14, abs=1e-15), k


def test_optional_families_are_off_by_default(orc):
    img = np.arange(64, dtype=np.uint16).reshape(8, 8)
    mask = np.ones((8, 8), dtype=np.int32)
    t = orc.extract(img, mask, 2, ng=8)
    assert not any(k.startswith(("GLRLM_", "GLSZM_")) for k in t)
    assert "GLDM_SDE" in t and "NGTDM_COARSENESS" in t


def test_glrlm_glszm_3d_closed_forms(orc):
    """3D: a constant line of L voxels along z is one run along the z axis
    and L runs of length 1 along each of the other 12 directions; a 3D
    checkerboard under 26-connectivity is two zones (the diagonal
    neighbours join each colour)."""
    L = 5
    img = np.full((7, 3, 3), 10, dtype=np.uint16)
    mask = np.zeros((7, 3, 3), dtype=np.int32)
    mask[1:1 + L, 1, 1] = 1
    t = _single(orc, img, mask, ndim=3, ng=4, families=("glrlm", "glszm"))
    assert t["GLRLM_RP"] == pytest.approx((1 / L + 12) / 13, rel=1e-14)
    assert t["GLRLM_LRE"] == pytest.approx((L ** 2 + 12) / 13, rel=1e-14)
    assert t["GLRLM_SRE"] == pytest.approx((1 / L ** 2 + 12) / 13, rel=1e-14)
    assert t["GLRLM_RLNU"] == pytest.approx((1 + 12 * L) / 13, rel=1e-14)
    assert t["GLSZM_ZP"] == pytest.approx(1 / L) and t["GLSZM_ZSM"] == L  # one zone
    n = 4
    zz, yy, xx = np.mgrid[0:n, 0:n, 0:n]
    img = ((xx + yy + zz) % 2).astype(np.uint16)
    mask = np.ones((n, n, n), dtype=np.int32)
    t = _single(orc, img, mask, ndim=3, ng=2, families=("glszm",))
    assert t["GLSZM_ZP"] == pytest.approx(2 / n ** 3) and t["GLSZM_ZSM"] == n ** 3 / 2
    assert t["GLSZM_ZE"] == pytest.approx(1.0) and t["GLSZM_GLM"] == pytest.approx(1.5)
