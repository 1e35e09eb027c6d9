"""GPU parity of the multi-block path (ROIs with more than 8192 pixels or a
padded bounding box above 16384 cells) against the FP64 oracle: 3D int16
volumes with 1e4-1.5e5-voxel ROIs, 2D uint16 ROIs whose bounding boxes span
several 65536-cell chunks, float batches (sorted order statistics), mixed
small/large batches, bit-exact co-occurrence counts and repeatability."""
import numpy as np
import pytest

import oracle
from paper_2603_12016_gb300 import workloads as W
from parity_util import compare, gpu_table, to_torch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BIG_PIX, BIG_CELLS, CHUNK = 8192, 16384, 65536


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()


def _dtype(a):
    return {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[a.dtype.type]


def _big_rows(t, ndim, pad):
    """Which oracle rows go to the multi-block class, and how many chunks the
    largest bounding box spans."""
    w, h = t["BBOX_WIDTH"], t["BBOX_HEIGHT"]
    d = t["BBOX_DEPTH"] if ndim == 3 else np.ones_like(w)
    padded = (w + 2 * pad) * (h + 2 * pad) * ((d + 2 * pad) if ndim == 3 else 1)
    big = (t["AREA"] > BIG_PIX) | (padded > BIG_CELLS)
    chunks = np.ceil(w * h * d / CHUNK).astype(int)
    return big, int(chunks[big].max()) if big.any() else 0


def _run(w, precision="fp32", per_offset=True, max_rois=256, features=None):
    from paper_2603_12016_gb300 import nyx

    prm = w.params
    ng = prm["glcm_levels"]
    ex = nyx.Extractor(w.image.shape, _dtype(w.image), ndim=w.ndim, glcm_levels=ng, dists=prm["dists"],
                       glcm_per_offset_cols=per_offset, hist_bins=prm["hist_bins"], precision=precision,
                       max_rois=max_rois, features=features)
    g = gpu_table(ex, to_torch(w.image), to_torch(w.mask))
    o = oracle.extract(w.image, w.mask, w.ndim, ng=max(ng, 2), dists=prm["dists"], hist_bins=prm["hist_bins"],
                       threads=8, families=("glrlm", "glszm"))
    return ex, g, o


def _assert_parity(g, o, ndim):
    fails = compare(g, o, ndim)
    assert not fails, "\n".join(fails[:40])


def _ct():
    return W.ct_3d(shape=(40, 128, 128), n_roi=6, seed=2301, vol_range=(9000, 150000))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_big_3d_int16(precision):
    w = _ct()
    ex, g, o = _run(w, precision)
    big, nch = _big_rows(o, 3, 1)
    assert big.sum() >= 4 and nch >= 2, (big.sum(), nch)
    _assert_parity(g, o, 3)


def test_big_2d_uint16_multichunk_two_distances():
    w = W.nuclei_2d(size=1024, n_roi=14, seed=2302, axis_range=(70.0, 190.0), min_px=50)
    ex, g, o = _run(w)
    big, nch = _big_rows(o, 2, 2)
    assert big.sum() >= 6 and nch >= 2, (big.sum(), nch)
    _assert_parity(g, o, 2)


def test_big_float_batch_sorted_order_stats():
    w = W.blob_batch_f32(batch=3, size=256, seed=2303, roi_range=(3, 6), px_range=(6000, 20000))
    w.params["glcm_levels"] = 16
    ex, g, o = _run(w)
    big, _ = _big_rows(o, 2, 1)
    assert big.sum() >= 4, big.sum()
    _assert_parity(g, o, 2)


def test_mixed_small_and_big_rois():
    """Every class in one call: warp, small, medium and multi-block ROIs."""
    w = W.blob_batch_f32(batch=4, size=256, seed=2304, roi_range=(8, 24), px_range=(30, 20000))
    w.params["glcm_levels"] = 32
    ex, g, o = _run(w)
    big, _ = _big_rows(o, 2, 1)
    assert big.sum() >= 2 and (~big).sum() >= 20, (big.sum(), (~big).sum())
    _assert_parity(g, o, 2)


def test_big_targeted_subset():
    """Only an order statistic and one texture feature selected: the
    geometry and centroid columns are still complete."""
    w = _ct()
    ex, g, o = _run(w, features=["MEDIAN", "GLCM_CONTRAST"], per_offset=False)
    assert "CENTROID_Z" in ex.columns and "VARIANCE" not in ex.columns
    _assert_parity(g, o, 3)


@pytest.mark.parametrize("features", [
    ["GLDM_SDE", "GLDM_GLN", "GLDM_DV", "GLDM_DE", "GLDM_LDHGLE"],
    ["GLDM_DN", "GLDM_GLV", "GLDM_SDLGLE", "NGTDM_COARSENESS", "NGTDM_STRENGTH"],
])
def test_big_gldm_without_glcm(features):
    """GLDM alone, and GLDM with NGTDM, on multi-block 3D ROIs: the
    neighbour kernel runs without the GLCM kernels."""
    w = _ct()
    ex, g, o = _run(w, features=features, per_offset=False)
    assert not any(c.startswith("GLCM_") for c in ex.columns)
    assert all(f in ex.columns for f in features)
    _assert_parity(g, o, 3)


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_big_glcm_counts_bit_exact(cfg):
    from paper_2603_12016_gb300 import nyx

    if cfg == "3d":
        w = _ct()
    else:
        w = W.nuclei_2d(size=1024, n_roi=14, seed=2302, axis_range=(70.0, 190.0), min_px=50)
    ng, dists = w.params["glcm_levels"], w.params["dists"]
    ex = nyx.Extractor(w.image.shape, _dtype(w.image), ndim=w.ndim, glcm_levels=ng, dists=dists, max_rois=256)
    img, mask = to_torch(w.image), to_torch(w.mask)
    lab, cnt = np.unique(w.mask[w.mask > 0], return_counts=True)
    ndirs = 13 if w.ndim == 3 else 4
    for row in (int(np.argmax(cnt)), int(np.argsort(cnt)[len(cnt) // 2])):
        ex.debug_select(row)
        ex(img, mask)
        key = oracle.roi_key(0, lab[row])
        for di, d in enumerate(dists):
            for k in range(ndirs):
                got = ex.debug_glcm(di * ndirs + k).astype(np.int64)
                ref = oracle.roi_glcm(w.image, w.mask, w.ndim, key, ng, k, d).astype(np.int64)
                assert np.array_equal(got, ref), (row, d, k)


def test_big_repeatable():
    """Multi-block merges run in chunk order: two calls give identical tables."""
    from paper_2603_12016_gb300 import nyx

    w = _ct()
    ex = nyx.Extractor(w.image.shape, torch.int16, ndim=3, glcm_levels=64, dists=(1,), max_rois=256)
    img, mask = to_torch(w.image), to_torch(w.mask)
    t1 = torch.empty((256, len(ex.columns)), dtype=torch.float64, device="cuda")
    t2 = torch.empty_like(t1)
    ex.extract_into(img, mask, t1)
    n = ex.extract_into(img, mask, t2)
    ex.sync_status()
    k = int(n.item())
    assert torch.equal(torch.nan_to_num(t1[:k], nan=-7.0), torch.nan_to_num(t2[:k], nan=-7.0))


def _sampled(w, ndim, rng_seed, n_random=8, features=None):
    """Full-size workload in the launch configuration of the benchmark,
    checked on a sample of ROIs the oracle computes one by one (the largest,
    the smallest and random ones)."""
    from paper_2603_12016_gb300 import nyx

    prm = w.params
    ng = prm["glcm_levels"]
    ex = nyx.Extractor(w.image.shape, _dtype(w.image), ndim=ndim, glcm_levels=ng, dists=prm["dists"],
                       glcm_per_offset_cols=False, hist_bins=prm["hist_bins"], max_rois=8192, features=features)
    g = gpu_table(ex, to_torch(w.image), to_torch(w.mask))
    keys = (g["IMAGE"].astype(np.int64) << 32) | g["LABEL"].astype(np.int64)
    order = np.argsort(g["AREA"])
    rng = np.random.default_rng(rng_seed)
    pick = set(order[:3].tolist()) | set(order[-3:].tolist()) | set(rng.choice(len(keys), n_random, replace=False).tolist())
    rows = np.array(sorted(pick))
    o = oracle.extract(w.image, w.mask, ndim, ng=max(ng, 2), dists=prm["dists"], hist_bins=prm["hist_bins"],
                       rois=[int(keys[i]) for i in rows], threads=8, families=("glrlm", "glszm"))
    g = {k: v[rows] for k, v in g.items()}
    return g, o


def test_ct3d_512x512x128_sampled():
    w = W.config("ct3d")
    g, o = _sampled(w, 3, 31)
    assert o["AREA"].max() > 5e5
    _assert_parity(g, o, 3)


def test_blobbatch_64x512_sampled():
    w = W.config("blobbatch")
    g, o = _sampled(w, 2, 32, n_random=16)
    assert o["AREA"].max() > 8192
    _assert_parity(g, o, 2)


def test_big_3d_wide_plane_global_neighbours():
    """A slab ROI with 300x300 planes: its one-plane halo does not fit beside
    the co-occurrence triangles in shared memory, so its spans read
    neighbours from global memory; a smaller ROI in the same volume takes the
    shared-memory raster path."""
    rng = np.random.default_rng(2306)
    img = rng.integers(-200, 1800, size=(8, 320, 320)).astype(np.int16)
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[2:6, 10:310, 12:312] = 3
    zz, yy, xx = np.ogrid[0:8, 0:320, 0:320]
    mask[((zz - 4) / 3.5) ** 2 + ((yy - 160) / 60.0) ** 2 + ((xx - 160) / 70.0) ** 2 <= 1.0] = 9
    w = W.Workload("slab3d", img, mask, 3, params=dict(glcm_levels=64, dists=(1,), hist_bins=256), meta={"n_roi": 2})
    ex, g, o = _run(w)
    assert list(g["LABEL"]) == [3, 9]
    _assert_parity(g, o, 3)
