"""The label scan's two staging paths: rows staged into shared memory by
bulk tensor copies (taken whenever both row pitches are multiples of 16
bytes) and rows loaded into registers (any width).  Both must give the
oracle's pixel counts, bounding boxes and intensity ranges bit for bit, and
the same table as each other (Extractor.set_scan_staging(1) selects the
register path)."""
import numpy as np
import pytest

import oracle
from parity_util import compare, gpu_table, to_torch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCAN_COLS = ("LABEL", "IMAGE", "AREA", "BBOX_XMIN", "BBOX_YMIN", "BBOX_ZMIN", "BBOX_WIDTH", "BBOX_HEIGHT",
             "BBOX_DEPTH", "MIN", "MAX")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()


def _case(shape, dtype, ndim, seed):
    """Blobs of many labels plus isolated single-pixel labels, so that tiles
    hold many labels and strips change label from row to row."""
    rng = np.random.default_rng(seed)
    if dtype == np.float32:
        img = rng.normal(100.0, 30.0, size=shape).astype(np.float32)
    elif dtype == np.int16:
        img = rng.integers(-1000, 3000, size=shape).astype(np.int16)
    else:
        img = rng.integers(0, 60000, size=shape).astype(np.uint16)
    mask = np.zeros(shape, dtype=np.int32)
    flat = mask.reshape(-1, shape[-2], shape[-1])
    lab = 1
    for pl in flat:
        for _ in range(12):
            h, w = rng.integers(2, 12), rng.integers(2, 40)
            y, x = rng.integers(0, shape[-2] - h), rng.integers(0, shape[-1] - w)
            pl[y:y + h, x:x + w] = lab if ndim == 2 else 1 + lab % 9
            lab += 1
        for _ in range(20):
            pl[rng.integers(0, shape[-2]), rng.integers(0, shape[-1])] = lab if ndim == 2 else 1 + lab % 9
            lab += 1
    return img, mask


SEEDS = {"u16_2d_200": 11, "i16_3d_136": 12, "f32_batch_260": 13, "u16_2d_204": 14}
CASES = {
    # 200 columns: one full 128-column tile and a partial one; 37 rows: a
    # ragged last tile and a last stage of one row
    "u16_2d_200": ((37, 200), np.uint16, 2),
    # 33-row planes: two-row stages cross plane boundaries
    "i16_3d_136": ((5, 33, 136), np.int16, 3),
    # a batch of three float images, 260 columns
    "f32_batch_260": ((3, 45, 260), np.float32, 2),
    # 204 columns: a 408-byte row pitch, so only the register path applies
    "u16_2d_204": ((40, 204), np.uint16, 2),
}

def _extract(img, mask, ndim, staging):
    from paper_2603_12016_gb300 import nyx

    dt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[img.dtype.type]
    ex = nyx.Extractor(img.shape, dt, ndim=ndim, glcm_levels=16, dists=(1,), max_rois=4096)
    ex.set_scan_staging(staging)
    assert ex.tuning()[5] == staging
    return gpu_table(ex, to_torch(img), to_torch(mask))


@pytest.mark.parametrize("name", sorted(CASES))
def test_scan_staging_paths_agree_with_oracle_and_each_other(name):
    shape, dtype, ndim = CASES[name]
    img, mask = _case(shape, dtype, ndim, seed=SEEDS[name])
    g = _extract(img, mask, ndim, 0)
    o = oracle.extract(img, mask, ndim, ng=16, dists=(1,), hist_bins=256, threads=8)
    n = len(o["LABEL"])
    assert len(g["LABEL"]) == n > 0
    for c in SCAN_COLS:
        if c in o:
            assert np.array_equal(g[c], o[c]), c
    fails = compare(g, o, ndim)
    assert not fails, "\n".join(fails[:20])
    # the same extraction with the register-load scan
    h = _extract(img, mask, ndim, 1)
    for c in SCAN_COLS:
        if c in g:
            assert np.array_equal(g[c], h[c]), c
    for c in g:  # downstream of the scan both paths stage the same pixels
        a, b = np.asarray(g[c], dtype=np.float64), np.asarray(h[c], dtype=np.float64)
        assert np.allclose(a, b, rtol=1e-6, atol=1e-9, equal_nan=True), c
