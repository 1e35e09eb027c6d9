"""GPU parity of the run-length (GLRLM) and size-zone (GLSZM) features:
crafted ROIs for the degenerate and extreme cases of runs and zones, the
same ROIs through the multi-block path, 3D volumes, float images, targeted
selections and run-to-run determinism, all against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from parity_util import compare, gpu_table, to_torch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RL = ["GLRLM_" + n for n in ("SRE", "LRE", "GLNU", "GLNUN", "RLNU", "RLNUN", "RP", "GLV", "RV", "RE", "LGLRE",
                             "HGLRE", "SRLGLE", "SRHGLE", "LRLGLE", "LRHGLE")]
SZ = ["GLSZM_" + n for n in ("SAE", "LAE", "GLNU", "GLNUN", "SZNU", "SZNUN", "ZP", "GLV", "ZV", "ZE", "LGLZE",
                             "HGLZE", "SALGLE", "SAHGLE", "LALGLE", "LAHGLE", "GLM", "ZSM")]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()


def _dt(a):
    return {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[a.dtype.type]


def _extract(img, mask, ndim, ng, limits=None, features=None, max_rois=1024):
    from paper_2603_12016_gb300 import nyx

    ex = nyx.Extractor(img.shape, _dt(img), ndim=ndim, glcm_levels=ng, dists=(1,), max_rois=max_rois,
                       features=features)
    if limits is not None:
        ex.set_class_limits(*limits)
    return ex, gpu_table(ex, to_torch(img), to_torch(mask))


def _check(img, mask, ndim, ng, limits=None, features=None):
    ex, g = _extract(img, mask, ndim, ng, limits, features)
    o = oracle.extract(img, mask, ndim, ng=ng, dists=(1,), threads=8, families=("glrlm", "glszm"))
    assert all(c in ex.columns for c in (features or RL + SZ) if c.startswith(("GLRLM_", "GLSZM_")))
    fails = compare(g, o, ndim)
    assert not fails, "\n".join(fails[:30])
    return g, o


def crafted_2d(seed=5):
    """ROIs that stress runs and zones: a single pixel, a uniform block (one
    zone, runs = its rows), long lines (runs longer than 1,000 px), a
    two-level checkerboard (two diagonal zones), a ring around a hole, an
    ROI on the image border, noise at many levels, and a thin diagonal."""
    rng = np.random.default_rng(seed)
    H, W = 384, 3200
    img = rng.integers(0, 4000, size=(H, W)).astype(np.uint16)
    mask = np.zeros((H, W), dtype=np.int32)
    mask[5, 5] = 1                                     # single pixel
    mask[10:40, 10:50] = 2
    img[10:40, 10:50] = 777                            # uniform: vmin == vmax
    mask[50, 10:1210] = 3                              # 1,200 px line
    img[50, 10:1210] = np.where(np.arange(1200) < 900, 100, 3000)  # a 900-run and a 300-run
    mask[60, 10:3010] = 4                              # 3,000 px line (large block class)
    img[60, 10:3010] = 1234
    yy, xx = np.mgrid[0:40, 0:40]
    mask[80:120, 10:50] = 5
    img[80:120, 10:50] = np.where((yy + xx) % 2 == 0, 10, 2000)  # checkerboard
    r = np.hypot(yy - 19.5, xx - 19.5)
    ring = (r > 8) & (r < 18)
    mask[130:170, 10:50][ring] = 6
    img[130:170, 10:50][ring] = rng.integers(0, 3, size=ring.sum()) * 1000
    mask[H - 30:H, W - 40:W] = 7                       # on the image border
    mask[200:260, 100:160] = 8                         # noise (many levels)
    for k in range(300):                               # diagonal line
        mask[70 + k // 4, 100 + k] = 9
    mask[300:340, 200:240] = 10
    img[300:340, 200:240] = (rng.integers(0, 4, size=(40, 40)) * 1000).astype(np.uint16)  # few levels, big zones
    return img, mask


@pytest.mark.parametrize("ng", [4, 64, 256])
def test_crafted_2d(ng):
    img, mask = crafted_2d()
    g, o = _check(img, mask, 2, ng)
    # the uniform block: one zone, each row one run (direction 0)
    row = int(np.flatnonzero(g["LABEL"] == 2)[0])
    assert g["GLSZM_ZP"][row] == 1.0 / 1200 and g["GLSZM_ZSM"][row] == 1200.0
    one = int(np.flatnonzero(g["LABEL"] == 1)[0])
    assert g["GLRLM_RP"][one] == 1.0 and g["GLSZM_ZE"][one] == 0.0


@pytest.mark.parametrize("limits", [(0, 0, 0, 0), (256, 0, 0, 0), (0, 1024, 0, 0)])
def test_crafted_2d_multiblock(limits):
    """The same ROIs through the multi-block kernels (runs walked and zones
    linked in global memory, across chunk boundaries)."""
    img, mask = crafted_2d()
    _check(img, mask, 2, 64, limits=limits)


def test_3d_volume_with_multiblock_rois():
    """Ellipsoids of up to ~60,000 voxels: 13 run directions, 26-connected
    zones, block and multi-block classes in one call."""
    from paper_2603_12016_gb300 import workloads as W

    w = W.ct_3d(shape=(48, 128, 128), n_roi=10, seed=77, vol_range=(300, 60000))
    ng = 16
    _, g = _extract(w.image, w.mask, 3, ng)
    assert g["AREA"].max() > 16384
    o = oracle.extract(w.image, w.mask, 3, ng=ng, dists=(1,), threads=8, families=("glrlm", "glszm"))
    fails = compare(g, o, 3)
    assert not fails, "\n".join(fails[:30])


def test_3d_crafted_lines_and_planes():
    rng = np.random.default_rng(9)
    img = rng.integers(0, 500, size=(20, 40, 40)).astype(np.int16) - 250
    mask = np.zeros(img.shape, dtype=np.int32)
    mask[2:18, 5, 5] = 1                   # line along z
    img[2:18, 5, 5] = 7
    mask[4, 2:38, 2:38] = 2                # a plane: one zone per level
    img[4, 2:38, 2:38] = (np.arange(36)[None, :] // 9 * 100).astype(np.int16)
    mask[8:16, 10:30, 10:30] = 3           # noise block
    mask[0, 0, 0] = 4                      # corner voxel
    for limits in (None, (0, 0, 0, 0)):
        _check(img, mask, 3, 8, limits=limits)


def test_float_batch():
    rng = np.random.default_rng(3)
    img = rng.normal(0, 1, size=(3, 96, 96)).astype(np.float32)
    img[1, 20:40, 20:40] = 0.5
    mask = np.zeros(img.shape, dtype=np.int32)
    for b in range(3):
        for k in range(9):
            y, x = 8 + 30 * (k // 3), 8 + 30 * (k % 3)
            mask[b, y:y + 20 + b, x:x + 18] = k + 1
    _check(img, mask, 2, 32)


@pytest.mark.parametrize("which", ["rl", "sz"])
def test_single_family_selection(which):
    img, mask = crafted_2d(seed=6)
    feats = RL if which == "rl" else SZ
    ex, _ = _extract(img, mask, 2, 32, features=feats)
    assert [c for c in ex.columns if c.startswith(("GLRLM_", "GLSZM_"))] == feats
    _check(img, mask, 2, 32, features=feats)


def test_runzone_columns_repeat_bit_for_bit():
    img, mask = crafted_2d(seed=8)
    for limits in (None, (0, 0, 0, 0)):
        ex, g1 = _extract(img, mask, 2, 64, limits)
        t = torch.stack([ex(to_torch(img), to_torch(mask)) for _ in range(3)])
        cols = [i for i, c in enumerate(ex.columns) if c.startswith(("GLRLM_", "GLSZM_"))]
        assert len(cols) == 34
        ref = t[0][:, cols]
        for k in range(1, 3):
            assert torch.equal(t[k][:, cols], ref)
