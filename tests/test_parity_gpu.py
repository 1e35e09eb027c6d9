"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs."""
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


def _nyx():
    from paper_2603_12016_gb300 import nyx

    return nyx


def _run(w, precision="fp32", per_offset=True, features=None, max_rois=None, rois=None):
    nyx = _nyx()
    prm = w.params
    ng = prm["glcm_levels"]
    ex = nyx.Extractor(w.image.shape, {np.uint16: torch.uint16, np.int16: torch.int16,
                                       np.float32: torch.float32}[w.image.dtype.type],
                       ndim=w.ndim, glcm_levels=ng, dists=prm["dists"], glcm_per_offset_cols=per_offset,
                       hist_bins=prm["hist_bins"], precision=precision, features=features,
                       max_rois=max_rois or max(1024, 2 * w.meta["n_roi"]))
    g = gpu_table(ex, to_torch(w.image), to_torch(w.mask))
    o = oracle.extract(w.image, w.mask, w.ndim, ng=max(ng, 2), dists=prm["dists"], hist_bins=prm["hist_bins"],
                       rois=rois, threads=8, families=("glrlm", "glszm"))
    if rois is not None:
        keys = (g["IMAGE"].astype(np.int64) << 32) | g["LABEL"].astype(np.int64)
        sel = np.isin(keys, np.array(sorted(rois), dtype=np.int64))
        g = {k: v[sel] for k, v in g.items()}
    return ex, g, o


def _assert_parity(g, o, ndim, **kw):
    fails = compare(g, o, ndim, **kw)
    assert not fails, "\n".join(fails[:40])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_blobs2d_256_full(precision):
    w = W.config("blobs2d")
    ex, g, o = _run(w, precision)
    assert len(g["LABEL"]) == w.meta["n_roi"] == 64
    _assert_parity(g, o, 2)


def test_nuclei2d_512_ng256_two_distances():
    w = W.config("nuclei2d_small")
    ex, g, o = _run(w)
    _assert_parity(g, o, 2)


def test_nuclei2d_2048_sampled():
    """Full-size 2048^2 / ~3600 ROIs / Ng 256 / d {1,2}: the launch the
    benchmark times, checked on a sample of ROIs the oracle computes one by
    one."""
    w = W.config("nuclei2d")
    rng = np.random.default_rng(7)
    labels = np.unique(w.mask[w.mask > 0])
    pick = rng.choice(labels, size=48, replace=False)
    # always include the largest and smallest ROIs
    lab, cnt = np.unique(w.mask[w.mask > 0], return_counts=True)
    pick = set(int(x) for x in pick) | {int(lab[np.argmax(cnt)]), int(lab[np.argmin(cnt)])}
    ex, g, o = _run(w, per_offset=False, rois=[oracle.roi_key(0, l) for l in pick], max_rois=8192)
    _assert_parity(g, o, 2)


def test_ct3d_small_i16():
    w = W.ct_3d(shape=(32, 96, 96), n_roi=12, seed=1203, vol_range=(200, 6000))
    ex, g, o = _run(w)
    _assert_parity(g, o, 3)


def test_blob_batch_f32():
    w = W.config("blobbatch_small")
    w.params["glcm_levels"] = 16
    ex, g, o = _run(w)
    _assert_parity(g, o, 2)


def test_targeted_subset_columns():
    w = W.config("blobs2d")
    feats = ["MEAN", "MEDIAN", "INT_HU", "GLCM_CONTRAST", "GLCM_CORR"]
    ex, g, o = _run(w, features=feats, per_offset=False)
    assert ex.columns[:11] == ["LABEL", "IMAGE", "AREA", "BBOX_XMIN", "BBOX_YMIN", "BBOX_WIDTH", "BBOX_HEIGHT",
                               "CENTROID_X", "CENTROID_Y", "MEAN", "MEDIAN"]
    assert "VARIANCE" not in ex.columns and "GLCM_CONTRAST_D1" in ex.columns and "INT_HU7" in ex.columns
    _assert_parity(g, o, 2)


GLDM_FEATURES = ["GLDM_" + f for f in ("SDE", "LDE", "GLN", "DN", "DNN", "GLV", "DV", "DE", "LGLE", "HGLE",
                                          "SDLGLE", "SDHGLE", "LDLGLE", "LDHGLE")]


@pytest.mark.parametrize("cfg,ng", [("blobs2d", 8), ("blobs2d", 256), ("blobbatch_small", 16)])
def test_gldm_only_selection(cfg, ng):
    """The GLDM selected alone (no GLCM, no NGTDM columns): the neighbour
    visit and the dependence counts run without the other texture groups,
    on integer and float images."""
    w = W.config(cfg)
    w.params["glcm_levels"] = ng
    ex, g, o = _run(w, features=GLDM_FEATURES, per_offset=False)
    assert [c for c in ex.columns if c.startswith("GLDM_")] == GLDM_FEATURES
    assert not any(c.startswith(("GLCM_", "NGTDM_")) for c in ex.columns)
    _assert_parity(g, o, w.ndim)


# ---------------------------------------------------------------------------
# bit-exact integer intermediates

def test_bins_bit_exact():
    w = W.config("nuclei2d_small")
    nyx = _nyx()
    ex = nyx.Extractor(w.image.shape, torch.uint16, glcm_levels=256, dists=(1, 2), max_rois=1024)
    bins = ex.debug_bins(to_torch(w.image), to_torch(w.mask)).cpu().numpy().astype(np.int64)
    labels = np.unique(w.mask[w.mask > 0])
    for lab in labels[:40]:
        ref = oracle.roi_bins(w.image, w.mask, 2, oracle.roi_key(0, lab), 256)
        got = bins[w.mask == lab]  # raster order = ascending linear index
        assert np.array_equal(got, ref), lab
    assert np.all(bins[w.mask == 0] == 0xFFFF)


@pytest.mark.parametrize("cfg", ["nuclei2d_small", "ct3d"])
def test_glcm_counts_bit_exact(cfg):
    nyx = _nyx()
    if cfg == "ct3d":
        w = W.ct_3d(shape=(24, 64, 64), n_roi=6, seed=77, vol_range=(300, 3000))
    else:
        w = W.config(cfg)
    ng = w.params["glcm_levels"]
    dists = w.params["dists"]
    dt = torch.uint16 if w.image.dtype == np.uint16 else torch.int16
    ex = nyx.Extractor(w.image.shape, dt, ndim=w.ndim, glcm_levels=ng, dists=dists, max_rois=1024)
    img, mask = to_torch(w.image), to_torch(w.mask)
    labels = np.unique(w.mask[w.mask > 0])
    ndirs = 13 if w.ndim == 3 else 4
    for row in (0, len(labels) // 2, len(labels) - 1):
        ex.debug_select(row)
        ex(img, mask)
        key = oracle.roi_key(0, labels[row])
        for di, d in enumerate(dists):
            for k in range(ndirs):
                got = ex.debug_glcm(di * ndirs + k).astype(np.int64)
                ref = oracle.roi_glcm(w.image, w.mask, w.ndim, key, ng, k, d).astype(np.int64)
                assert np.array_equal(got, ref), (row, d, k)


# ---------------------------------------------------------------------------
# edge cases

def test_edge_cases_2d():
    img = np.zeros((37, 41), dtype=np.uint16)  # width not a multiple of 4
    mask = np.zeros((37, 41), dtype=np.int32)
    rng = np.random.default_rng(3)
    img[:] = rng.integers(0, 4000, size=img.shape)
    mask[0, 0] = 5                       # single pixel in a corner
    mask[10:14, 40] = 2_000_000_000      # large label on the right border, 1 px wide
    mask[20:23, 5:9] = 7
    img[20:23, 5:9] = 1234               # constant ROI
    mask[30:37, 0:41] = 9                # full-width band on the bottom border
    mask[2, 2:30:3] = 11                 # disconnected pixels, no neighbour pairs
    w = W.Workload("edges", img, mask, 2, params=dict(glcm_levels=8, dists=(1, 2), hist_bins=16),
                   meta={"n_roi": 5})
    ex, g, o = _run(w)
    assert list(g["LABEL"]) == [5, 7, 9, 11, 2_000_000_000]
    _assert_parity(g, o, 2)
    assert np.isnan(g["GLCM_ASM_D1"][0]) and np.isnan(g["GLCM_ASM_D1"][3])


def test_empty_mask_and_errors():
    nyx = _nyx()
    img = torch.zeros((16, 16), dtype=torch.uint16, device="cuda")
    mask = torch.zeros((16, 16), dtype=torch.int32, device="cuda")
    ex = nyx.Extractor((16, 16), torch.uint16, glcm_levels=8, max_rois=64)
    assert ex(img, mask).shape[0] == 0
    assert ex.count_rois(img, mask) == 0
    mask[3, 3] = -1
    with pytest.raises(nyx.NyxError) as e:
        ex(img, mask)
    assert e.value.status == 4
    mask[3, 3] = 0
    mask[0, :] = torch.arange(1, 17, dtype=torch.int32)
    with pytest.raises(nyx.NyxError) as e:  # 16 ROIs, room for 8
        ex(img, mask, cap=8)
    assert e.value.status == 6
    assert ex(img, mask).shape[0] == 16  # the plan recovers after an error
    f = nyx.Extractor((16, 16), torch.float32, glcm_levels=8, max_rois=64)
    fimg = torch.ones((16, 16), dtype=torch.float32, device="cuda")
    fimg[0, 4] = float("nan")
    with pytest.raises(nyx.NyxError) as e:
        f(fimg, mask)
    assert e.value.status == 5
    with pytest.raises(nyx.NyxError):
        nyx.Extractor((16, 16), torch.uint16, glcm_levels=300)


def test_repeatable_and_sync_free_launches():
    """Back-to-back asynchronous extractions on one stream give identical
    tables (no state leaks between calls)."""
    nyx = _nyx()
    w = W.config("nuclei2d_small")
    ex = nyx.Extractor(w.image.shape, torch.uint16, glcm_levels=256, dists=(1, 2), max_rois=1024)
    img, mask = to_torch(w.image), to_torch(w.mask)
    t1 = torch.empty((1024, len(ex.columns)), dtype=torch.float64, device="cuda")
    t2 = torch.empty_like(t1)
    ex.extract_into(img, mask, t1)
    n = ex.extract_into(img, mask, t2)
    ex.sync_status()
    k = int(n.item())
    assert torch.equal(torch.nan_to_num(t1[:k], nan=-7.0), torch.nan_to_num(t2[:k], nan=-7.0))


# ---------------------------------------------------------------------------
# CUDA-graph replay and size-class limits

def test_graph_replay_matches_direct_launches():
    nyx = _nyx()
    w = W.config("nuclei2d_small")
    img, mask = to_torch(w.image), to_torch(w.mask)
    ex = nyx.Extractor(w.image.shape, torch.uint16, glcm_levels=256, dists=(1, 2), max_rois=1024)
    t = [torch.full((1024, len(ex.columns)), -1.0, dtype=torch.float64, device="cuda") for _ in range(3)]
    n = ex.extract_into(img, mask, t[0])
    ex.extract_into(img, mask, t[0])          # same arguments: replay
    assert ex.graph_captures() == 1
    ex.extract_into(img, mask, t[1])          # new table pointer: second graph
    assert ex.graph_captures() == 2
    ex.extract_into(img, mask, t[0])          # both stay cached
    assert ex.graph_captures() == 2
    ex.sync_status()
    ex.use_graphs(False)
    ex.extract_into(img, mask, t[2])
    ex.sync_status()
    k = int(n.item())
    ref = torch.nan_to_num(t[2][:k], nan=-7.0)
    for tt in t[:2]:
        assert torch.equal(torch.nan_to_num(tt[:k], nan=-7.0), ref)


@pytest.mark.parametrize("limits", [None, (0, 0, 4096, 0), (128, 0, 0, 8192), (256, 1024, 0, 0), (0, 512, 2048, 8192),
                                    (64, 512, 2048, 0, 8), (256, 1024, 4096, 8192, 32), (0, 1024, 4096, 0, 16, 1),
                                    (0, 0, 0, 0)])
def test_class_limits_and_autotune_keep_parity(limits):
    """Any class limits (autotuned or set) route ROIs to other kernels; the
    table must still match the oracle.  (256, 1024, 0, 0) sends every ROI
    above 1,024 px to the multi-block path, (0, 0, 0, 0) every ROI."""
    nyx = _nyx()
    w = W.config("nuclei2d_small")
    img, mask = to_torch(w.image), to_torch(w.mask)
    ex = nyx.Extractor(w.image.shape, torch.uint16, glcm_levels=256, dists=(1, 2), max_rois=1024)
    if limits is None:
        lim = ex.autotune(img, mask, reps=2)
        assert lim[0] in (0, 64, 128, 256) and lim[1] in (0, 512, 1024) and lim[2] in (0, 2048, 4096)
        assert lim[3] in (0, 8192) and lim[4] in (8, 16, 32) and lim[5] in (0, 1) and ex.tuning() == lim
    elif len(limits) >= 5:  # class limits, the label scan's tile height [and row staging]
        ex.set_tuning(*limits)
        assert ex.tuning() == (limits + (0,))[:6]
    else:
        ex.set_class_limits(*limits)
    g = gpu_table(ex, img, mask)
    o = oracle.extract(w.image, w.mask, 2, ng=256, dists=(1, 2), hist_bins=256, threads=8, families=("glrlm", "glszm"))
    _assert_parity(g, o, 2)


@pytest.mark.parametrize("case", ["bitmap_high_base", "bit16_boundary", "wide_31bit", "batch2"])
def test_key_sort_paths(case):
    """ROI rows come out in ascending (image, label) order on both key-sort
    paths: the presence bitmap (keys differing in their low 16 bits only,
    here based at 0x30000) and the radix sort (wider label ranges, batches).
    Areas and bounding boxes are checked against numpy, the full feature
    set against the oracle."""
    rng = np.random.default_rng({"bitmap_high_base": 41, "bit16_boundary": 42, "wide_31bit": 43, "batch2": 44}[case])
    nb = 2 if case == "batch2" else 1
    img = rng.integers(0, 3000, size=(nb, 96, 96)).astype(np.uint16)
    mask = np.zeros(img.shape, dtype=np.int32)
    n = 180
    if case == "bitmap_high_base":
        labels = rng.choice(np.arange(0x30000, 0x40000), size=n, replace=False)
        labels[:2] = [0x30000, 0x3FFFF]
    elif case == "bit16_boundary":
        labels = rng.choice(np.arange(60000, 70000), size=n, replace=False)
        labels[:2] = [65535, 65536]
    else:
        labels = rng.choice(np.arange(1, 2**31 - 1, 9973), size=n, replace=False)
    slots = rng.permutation(32 * 32)[:n]
    for lab, sl in zip(labels, slots):
        b = int(rng.integers(0, nb))
        y, x = 3 * (sl // 32), 3 * (sl % 32)
        mask[b, y:y + 2, x:x + 1 + int(rng.integers(1, 3))] = lab
    if nb == 1:
        img, mask = img[0], mask[0]
    w = W.Workload(case, img, mask, 2, params=dict(glcm_levels=16, dists=(1,), hist_bins=16), meta={"n_roi": n})
    ex, g, o = _run(w, max_rois=1024)
    bi = np.nonzero(mask)[0] if nb > 1 else np.zeros(np.count_nonzero(mask), dtype=np.int64)
    keys = np.unique((bi.astype(np.int64) << 32) | mask[mask > 0].astype(np.int64))
    got = (g["IMAGE"].astype(np.int64) << 32) | g["LABEL"].astype(np.int64)
    assert np.array_equal(got, keys)
    for k, area in zip(keys, g["AREA"]):
        m = (mask[k >> 32] if nb > 1 else mask) == (k & 0xFFFFFFFF)
        assert area == m.sum()
    _assert_parity(g, o, 2)


@pytest.mark.parametrize("ndim", [2, 3])
def test_signed_intensities_summing_near_zero(ndim):
    """int16 ROIs whose intensities nearly cancel (CT values around 0 HU) put
    the intensity-weighted centroid far outside the ROI: the raw and central
    intensity moments must still match the FP64 definition, and eta with a
    negative total intensity is NaN wherever the normalising power is not
    real."""
    nyx = _nyx()
    rng = np.random.default_rng(61 + ndim)
    shape = (96, 96) if ndim == 2 else (16, 48, 48)
    img = rng.integers(-250, 251, size=shape).astype(np.int16)
    mask = np.zeros(shape, dtype=np.int32)
    if ndim == 2:
        for k in range(9):
            y, x = 4 + 30 * (k // 3), 4 + 30 * (k % 3)
            mask[y:y + 22, x:x + 20 + k] = k + 1
        mask[0, 0] = 10
    else:
        mask[2:14, 4:22, 4:22] = 1
        mask[2:14, 26:44, 26:44] = 2
        mask[0, 0, 0] = 3
        img[0, 0, 0] = -17
    ex = nyx.Extractor(shape, torch.int16, ndim=ndim, glcm_levels=16, dists=(1,), max_rois=64)
    g = gpu_table(ex, to_torch(img), to_torch(mask))
    o = oracle.extract(img, mask, ndim, ng=16, dists=(1,), threads=8, families=("glrlm", "glszm"))
    _assert_parity(g, o, ndim)
