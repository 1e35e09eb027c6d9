"""Parity over the hyperparameter space the benchmarks do not visit: GLCM
grey levels 2..64, distances up to 8, histogram bins 2..4096, per-offset
columns in 3D, int16 2D images, batches of several 2D uint16 images, and the
FP64 path, each against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2603_12016_gb300 import workloads as W
from parity_util import compare, gpu_table, to_torch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()


def _dt(a):
    return {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[a.dtype.type]


def _check(img, mask, ndim, ng, dists, hist_bins, per_offset=True, precision="fp32", max_rois=1024):
    from paper_2603_12016_gb300 import nyx

    ex = nyx.Extractor(img.shape, _dt(img), ndim=ndim, glcm_levels=ng, dists=dists, glcm_per_offset_cols=per_offset,
                       hist_bins=hist_bins, precision=precision, max_rois=max_rois)
    g = gpu_table(ex, to_torch(img), to_torch(mask))
    o = oracle.extract(img, mask, ndim, ng=max(ng, 2), dists=dists, hist_bins=hist_bins, threads=8,
                       families=("glrlm", "glszm"))
    fails = compare(g, o, ndim)
    assert not fails, "\n".join(fails[:30])
    return ex, g


@pytest.mark.parametrize("ng,dists,hist_bins", [(2, (1,), 2), (7, (1, 3, 8), 13), (64, (2, 5), 4096)])
def test_2d_levels_distances_bins(ng, dists, hist_bins):
    w = W.config("nuclei2d_small")
    _check(w.image, w.mask, 2, ng, dists, hist_bins)


def test_3d_per_offset_two_distances():
    w = W.ct_3d(shape=(24, 64, 64), n_roi=8, seed=2501, vol_range=(300, 9000))
    ex, g = _check(w.image, w.mask, 3, 16, (1, 2), 32, per_offset=True)
    assert "GLCM_CONTRAST_D2_O12" in ex.columns


def test_int16_2d_negative_values():
    rng = np.random.default_rng(2502)
    w = W.config("nuclei2d_small")
    img = (w.image.astype(np.int32) - 20000).clip(-32768, 32767).astype(np.int16)
    img[rng.random(img.shape) < 0.01] = -32768
    _check(img, w.mask, 2, 32, (1,), 64)


def test_uint16_batch_of_images():
    imgs, masks = [], []
    for k in range(3):
        w = W.nuclei_2d(size=256, n_roi=40, seed=2510 + k)
        imgs.append(w.image)
        masks.append(w.mask)
    img, mask = np.stack(imgs), np.stack(masks)
    ex, g = _check(img, mask, 2, 32, (1, 2), 128)
    assert sorted(set(g["IMAGE"].astype(int).tolist())) == [0, 1, 2]


def test_fp64_path_3d_and_float():
    w = W.ct_3d(shape=(24, 64, 64), n_roi=6, seed=2503, vol_range=(300, 9000))
    _check(w.image, w.mask, 3, 32, (1,), 256, per_offset=False, precision="fp64")
    b = W.config("blobbatch_small")
    _check(b.image, b.mask, 2, 16, (1,), 256, per_offset=False, precision="fp64")


def _disc_image(size, rois, seed, dtype=np.uint16):
    """Discs of given (cy, cx, r, lo, hi): uniform values in [lo, hi)."""
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 1000, size=(size, size)).astype(np.int64)
    mask = np.zeros((size, size), dtype=np.int32)
    yy, xx = np.mgrid[0:size, 0:size]
    for k, (cy, cx, r, lo, hi) in enumerate(rois, start=1):
        inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
        mask[inside] = k
        img[inside] = rng.integers(lo, hi, size=int(inside.sum()))
    return img.astype(dtype), mask


def test_big_value_histogram_global_and_sorted_paths():
    """uint16 multi-block ROIs: a dense value range above the shared-memory
    histogram (global histogram), a range wider than the pixel count (sorted
    values), and a narrow one (shared-memory histogram)."""
    img, mask = _disc_image(512, [(130, 130, 110, 0, 20000),      # ~38K px, range 20K: global histogram
                                  (380, 380, 100, 0, 65536),      # ~31K px, range 65K > n: sorted values
                                  (130, 390, 80, 5000, 5300)], 2601)  # ~20K px, range 300: shared histogram
    _check(img, mask, 2, 64, (1, 2), 256, max_rois=64)


def test_big_2d_long_distances_multispan():
    img, mask = _disc_image(768, [(380, 380, 300, 0, 4000), (80, 80, 60, 100, 900)], 2602)
    _check(img, mask, 2, 32, (1, 4, 8), 64, per_offset=True, max_rois=64)


def test_big_float_3d():
    w = W.ct_3d(shape=(32, 96, 96), n_roi=5, seed=2603, vol_range=(9000, 40000))
    img = (w.image.astype(np.float32) * np.float32(0.37) + np.float32(12.5))
    _check(img, w.mask, 3, 24, (1,), 100, per_offset=False, max_rois=64)


def test_int16_big_2d_negative():
    img, mask = _disc_image(512, [(250, 250, 200, -30000, 30000)], 2604, dtype=np.int64)
    img = img.astype(np.int16)
    _check(img, mask, 2, 48, (1,), 256, max_rois=64)
