"""C-ABI checks that need no GPU: the library builds and loads, exports
every function include/nyx.h declares, and its host-only calls behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nyxlib():
    from paper_2603_12016_gb300 import build

    build.build()
    from paper_2603_12016_gb300 import nyx

    return nyx


def _declared():
    src = open(os.path.join(ROOT, "include", "nyx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nyx_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("nyx_create", "nyx_plan_create", "nyx_extract", "nyx_count_rois", "nyx_backward",
                 "nyx_num_columns", "nyx_column_name", "nyx_sync_status", "nyx_debug_glcm", "nyx_debug_bins"):
        assert must in names


def test_library_exports_every_declared_symbol(nyxlib):
    L = nyxlib.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_feature_ids(nyxlib):
    fid = nyxlib.feature_id
    assert fid("MEAN") == 0 and fid("UNIFORMITY") == 40
    assert fid("INT_M") == 41 and fid("BIN_HU") == 50
    assert fid("GLCM_ASM") == 51 and fid("GLCM_VARIANCE") == 80
    assert fid("EDGE_INTEGRATED_INTENSITY") == 81 and fid("EDGE_STDDEV_INTENSITY") == 85
    assert fid("NGTDM_COARSENESS") == 86 and fid("NGTDM_STRENGTH") == 90
    assert fid("GLDM_SDE") == 91 and fid("GLDM_LDHGLE") == 104
    assert fid("GLRLM_SRE") == 105 and fid("GLRLM_LRHGLE") == 120
    assert fid("GLSZM_SAE") == 121 and fid("GLSZM_ZSM") == 138
    assert fid("NOPE") == -1
    ids = [fid(n) for n in ("MEAN", "INT_HU", "GLCM_CORR")]
    assert len(set(ids)) == 3


def test_params_default_and_validation(nyxlib):
    L = nyxlib.lib()
    p = nyxlib.NyxParams()
    assert L.nyx_params_default(ctypes.byref(p), 640, 480) == 0
    assert p.struct_size == ctypes.sizeof(nyxlib.NyxParams)
    assert (p.dims[0], p.dims[1], p.dims[2], p.ndim, p.batch) == (640, 480, 1, 2, 1)
    assert p.glcm_levels == 64 and p.hist_bins == 256 and all(m == 2 ** 64 - 1 for m in p.feature_mask)
    # a null context is rejected before any device call
    assert L.nyx_plan_create(None, ctypes.byref(p), ctypes.byref(ctypes.c_void_p())) == 1
    assert L.nyx_create(None, 0) == 1
    assert L.nyx_extract(None, None, None, None, 0, None, 0, None) == 1


GEOMETRY = {"LABEL", "IMAGE", "AREA", "BBOX_XMIN", "BBOX_YMIN", "BBOX_ZMIN", "BBOX_WIDTH", "BBOX_HEIGHT", "BBOX_DEPTH",
            "CENTROID_X", "CENTROID_Y", "CENTROID_Z"}


def _feature_of_column(col):
    """The feature name a table column belongs to: GLCM columns carry a
    distance (and an offset) suffix, moment columns their indices."""
    m = re.match(r"(GLCM_[A-Z0-9]+)_D\d+(_[AO]\d+)?$", col)
    if m:
        return m.group(1)
    m = re.match(r"((INT|BIN)_(M|MU|ETA|NU|HU))\d+$", col)
    if m:
        return m.group(1)
    return col


@pytest.mark.parametrize("ndim", [2, 3])
def test_oracle_and_library_share_the_feature_registry(nyxlib, ndim):
    """Every feature column of the oracle maps to a library feature id, and
    every library feature id has an oracle column: the two sides agree on
    the feature set by name, without a GPU."""
    import numpy as np

    import oracle

    shape = (6, 6) if ndim == 2 else (3, 4, 4)
    img = np.arange(int(np.prod(shape)), dtype=np.uint16).reshape(shape)
    t = oracle.extract(img, np.ones(shape, dtype=np.int32), ndim, ng=8, dists=(1, 2), families=("glrlm", "glszm"))
    ids = set()
    for col in t:
        if col in GEOMETRY:
            continue
        fid = nyxlib.feature_id(_feature_of_column(col))
        assert fid >= 0, col
        ids.add(fid)
    # 2D has no z centroid; 3D moments have no normalised-raw and Hu families
    absent = {nyxlib.feature_id("WEIGHTED_CENTROID_Z")} if ndim == 2 else \
        {nyxlib.feature_id(n) for n in ("INT_NU", "INT_HU", "BIN_NU", "BIN_HU")}
    assert ids == set(range(139)) - absent
