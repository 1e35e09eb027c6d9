"""Soft-feature planning: the Eq. 8 separability ratio (pinned to the one-way
ANOVA F statistic, which is the same quantity), the Eq. 5 ordering check,
and on the GPU the timing grid over grey depth x nested distance sets and
the separability grid on labelled texture classes."""
import math

import numpy as np
import pytest
import scipy.stats

from paper_2603_12016_gb300 import softgrid
from paper_2603_12016_gb300 import workloads as W


@pytest.mark.parametrize("seed,k", [(1, 2), (2, 3), (3, 5)])
def test_f_ratio_is_one_way_anova_f(seed, k):
    rng = np.random.default_rng(seed)
    groups = [rng.normal(loc=0.3 * i, scale=1.0 + 0.2 * i, size=int(rng.integers(5, 40))) for i in range(k)]
    v = np.concatenate(groups)
    c = np.concatenate([np.full(g.size, i) for i, g in enumerate(groups)])
    perm = rng.permutation(v.size)
    got = softgrid.f_ratio(v[perm], c[perm])
    assert got == pytest.approx(scipy.stats.f_oneway(*groups).statistic, rel=1e-12)


def test_f_ratio_hand_computed_and_degenerate():
    # classes {1, 3} and {5, 7}: grand mean 4, between = 2*1 + 2*1... written out:
    # n_i (m_i - m)^2 = 2*(2-4)^2 + 2*(6-4)^2 = 16; within = 4 * 1 = 4; (N-K)/(K-1) = 2
    assert softgrid.f_ratio([1, 3, 5, 7], [0, 0, 1, 1]) == pytest.approx(2 * 16 / 4)
    assert math.isnan(softgrid.f_ratio([1, 2, 3], [0, 0, 0]))          # one class
    assert math.isnan(softgrid.f_ratio([1, 1, 5, 5], [0, 0, 1, 1]))    # no within-class spread
    # non-finite values and unlabelled samples (class -1) are left out
    assert softgrid.f_ratio([1, 3, np.nan, 5, 7, 100], [0, 0, 0, 1, 1, -1]) == pytest.approx(8.0)


def test_monotone_report():
    t = np.array([[1.0, 2.0, 3.0], [1.5, 2.5, 3.5]])
    r = softgrid.monotone_report(t)
    assert r["steps"] == 7 and r["holds"] == 7 and not r["violations"]
    t[1, 1] = 1.4   # faster than its left neighbour and than the point above
    r = softgrid.monotone_report(t)
    assert r["holds"] == 5 and {v[0] for v in r["violations"]} == {"levels", "dists"}
    assert softgrid.monotone_report(t, rel_tol=0.5)["holds"] == 7


def test_texture_classes_generator():
    w = W.texture_classes_2d(size=256, n_roi=60, seed=7)
    labels = np.unique(w.mask[w.mask > 0])
    cls = w.meta["classes"][labels]
    assert np.all(cls >= 0) and set(cls.tolist()) == {0, 1, 2}
    assert w.image.dtype == np.uint16 and w.meta["n_roi"] == labels.size


@pytest.mark.gpu
def test_timing_grid_ordered_over_distance_sets_and_levels():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()
    w = W.config("nuclei2d")
    t = softgrid.timing_grid(w, [16, 64, 256], [[1], [1, 2], [1, 2, 3, 4]], steps=10)
    r = softgrid.monotone_report(t, rel_tol=0.03)  # 3% for timing noise between neighbours
    assert r["holds"] == r["steps"], (t, r["violations"])
    assert t[-1, -1] > 1.5 * t[0, 0]  # four distances at Ng 256 cost well above one at Ng 16


@pytest.mark.gpu
def test_separability_grid_and_oracle_agree():
    """The Eq. 8 ratio of a GLCM feature on the GPU table equals the ratio on
    the oracle's table (the features agree within their tolerance), and the
    texture classes are separable by some GLCM feature."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2603_12016_gb300 import build, nyx

    build.build()
    w = W.texture_classes_2d(size=384, n_roi=120, seed=1106)
    sep = softgrid.separability_grid(w, w.meta["classes"], [32, 64], [[1], [1, 2]], max_rois=1024)
    best = max(v["ratio"] for v in sep["best_point"].values())
    assert best > 5.0, best
    ex = nyx.Extractor(w.image.shape, torch.uint16, glcm_levels=32, dists=(1,), max_rois=1024,
                       features=["GLCM_" + f for f in softgrid.GLCM_FEATURES])
    g = ex(torch.from_numpy(w.image).cuda(), torch.from_numpy(w.mask).cuda()).cpu().numpy()
    cols = {c: i for i, c in enumerate(ex.columns)}
    o = oracle.extract(w.image, w.mask, 2, ng=32, dists=(1,), threads=8)
    cls = w.meta["classes"][o["LABEL"].astype(np.int64)]
    for f in ("CONTRAST", "ENTROPY", "HOM1", "CORR"):
        rg = softgrid.f_ratio(g[:, cols[f"GLCM_{f}_D1"]], cls)
        ro = softgrid.f_ratio(o[f"GLCM_{f}_D1"], cls)
        assert rg == pytest.approx(ro, rel=1e-3), f
        assert rg == pytest.approx(sep["ratio"][f][0][0], rel=1e-9), f
