"""The seeded synthetic inputs that stand in for the paper's datasets: each
generator realises the shapes, pixel types, ROI counts and size ranges its
workload is described with, reproducibly, and the streamed mosaic's tiles
agree with the assembled image wherever they are cut.  No GPU."""
import numpy as np
import pytest

from paper_2603_12016_gb300 import workloads as W


def _sizes(mask):
    c = np.bincount(mask.ravel())[1:]
    return c[c > 0]


def test_blobs2d_recipe():
    w = W.config("blobs2d")
    assert w.image.shape == (256, 256) and w.image.dtype == np.uint16 and w.mask.dtype == np.int32
    s = _sizes(w.mask)
    assert s.size == w.meta["n_roi"] == 64
    assert s.min() >= 50 and s.max() <= 1500
    assert w.params["glcm_levels"] == 32 and tuple(w.params["dists"]) == (1,)


def test_nuclei2d_recipe_and_reproducibility():
    w = W.config("nuclei2d")
    assert w.image.shape == (2048, 2048) and w.image.dtype == np.uint16
    s = _sizes(w.mask)
    assert s.size == w.meta["n_roi"] == 3610
    assert s.min() >= 50 and s.max() <= 5000
    salt = np.mean(w.image == 65535)
    assert 0.015 < salt < 0.025  # 2% salt noise
    assert w.params["glcm_levels"] == 256 and tuple(w.params["dists"]) == (1, 2)
    v = W.config("nuclei2d")
    assert np.array_equal(w.image, v.image) and np.array_equal(w.mask, v.mask)
    u = W.config("nuclei2d", seed_offset=1)
    assert not np.array_equal(w.mask, u.mask)


def test_blobbatch_recipe():
    w = W.config("blobbatch")
    assert w.image.shape == (64, 512, 512) and w.image.dtype == np.float32 and w.ndim == 2
    per = [_sizes(m) for m in w.mask]
    n = [p.size for p in per]
    assert min(n) >= 4 and max(n) <= 256 and sum(n) == 2960
    allsz = np.concatenate(per)
    assert allsz.max() <= 20000
    cover = [(m > 0).mean() for m in w.mask]
    assert max(cover) <= 0.70 + 1e-9


def test_ct3d_recipe():
    w = W.config("ct3d")
    assert w.image.shape == (128, 512, 512) and w.image.dtype == np.int16 and w.ndim == 3
    assert w.image.min() >= -1000 and w.image.max() <= 3000
    s = _sizes(w.mask)
    assert s.size == w.meta["n_roi"] == 200
    assert 900 <= s.min() <= 1100 and 0.9e6 <= s.max() <= 1.1e6  # one ROI forced to each end
    assert 0.6 < (w.mask > 0).mean() < 0.9
    assert w.params["glcm_levels"] == 64 and tuple(w.params["dists"]) == (1,)


@pytest.mark.parametrize("win", [(0, 0, 512, 512), (300, 190, 700, 450), (1500, 1700, 548, 348)])
def test_mosaic_tiles_agree_with_the_assembled_image(win):
    """Any window generated on its own (tiles of any size, at any offset)
    equals the same window of the assembled mosaic: ROIs that cross tile
    borders and the hashed background are generated consistently."""
    m = W.mosaic_2d(size=2048, tile=512, n_roi=2000)
    img, mask = m.assemble()
    x0, y0, tw, th = win
    ti, tm = m.tile(x0, y0, tw, th)
    assert np.array_equal(ti, img[y0:y0 + th, x0:x0 + tw])
    assert np.array_equal(tm, mask[y0:y0 + th, x0:x0 + tw])


def test_mosaic_small_recipe():
    w = W.mosaic_workload("mosaic_small", 0, 1)
    assert w.image.shape == (8192, 8192) and w.image.dtype == np.uint16
    s = _sizes(w.mask)
    assert s.size == w.meta["n_roi"] and 20_000 < s.size <= 32_000
    assert s.max() <= 10_000  # areas drawn in [20, 1e4]; overwrites only shrink them
    assert w.meta["tile"] == 1024
