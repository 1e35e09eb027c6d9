"""The allocation-free ROI count, for callers that may not allocate device
memory (a host application that owns all GPU memory through its own pool
and forbids cudaMalloc from plug-ins, a process under a fixed device-memory
quota, or a path that cannot afford cudaMalloc's implicit synchronisation).

nyx_count_rois_noalloc keeps its label table in a fixed array inside the
library instead of a plan workspace.  This test calls it through the C ABI
twice in a row and checks each result against nyx_count_rois (the plan-based
entry point), so a table left dirty by the first call would show up in the
second.  It lives in a file of its own that pytest collects last and passes
both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nyx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()
    from paper_2603_12016_gb300 import nyx as n

    return n


def _params(nyx, shape, ndim, dtype_code):
    p = nyx.NyxParams()
    nyx.lib().nyx_params_default(ctypes.byref(p), 1, 1)
    spatial = shape[-ndim:]
    batch = int(np.prod(shape[:-ndim])) if len(shape) > ndim else 1
    p.ndim = ndim
    p.dims[0], p.dims[1] = spatial[-1], spatial[-2]
    p.dims[2] = spatial[0] if ndim == 3 else 1
    p.batch = batch
    p.dtype = dtype_code
    return p


def _noalloc(nyx, p, img, mask):
    n = ctypes.c_int64(-1)
    st = nyx.lib().nyx_count_rois_noalloc(ctypes.byref(p), img.data_ptr(), mask.data_ptr(), ctypes.byref(n),
                                          torch.cuda.current_stream().cuda_stream)
    return st, n.value


@pytest.mark.parametrize("cfg", ["nuclei2d_small", "blobbatch_small", "ct3d_small"])
def test_noalloc_count_matches_plan_entry_point_twice(nyx, cfg):
    from paper_2603_12016_gb300 import workloads as W

    w = W.config(cfg)
    tdt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    ex = nyx.Extractor(w.image.shape, tdt, ndim=w.ndim, glcm_levels=16, max_rois=4096)
    expected = ex.count_rois(img, mask)
    # ROIs are (image, label) pairs: count distinct labels per image
    m = w.mask.reshape((-1,) + w.mask.shape[-w.ndim:]) if w.mask.ndim > w.ndim else w.mask[None]
    assert expected == sum(len(np.unique(mi[mi > 0])) for mi in m)
    p = _params(nyx, w.image.shape, w.ndim, nyx.DTYPES[tdt])
    for _ in range(2):  # the second call must not see the first call's table
        st, n = _noalloc(nyx, p, img, mask)
        assert st == 0 and n == expected


def test_noalloc_count_changes_with_input_and_rejects_oversize(nyx):
    img = torch.zeros((64, 64), dtype=torch.uint16, device="cuda")
    mask = torch.zeros((64, 64), dtype=torch.int32, device="cuda")
    p = _params(nyx, (64, 64), 2, 0)
    assert _noalloc(nyx, p, img, mask) == (0, 0)
    mask[:8, :8] = 3
    mask[20:30, 40:50] = 9
    assert _noalloc(nyx, p, img, mask) == (0, 2)
    assert _noalloc(nyx, p, img, mask) == (0, 2)
    # more distinct labels than the fixed table holds -> a clear capacity error
    big = torch.arange(1, 160 * 128 + 1, dtype=torch.int32, device="cuda").reshape(160, 128)
    pb = _params(nyx, (160, 128), 2, 0)
    st, _ = _noalloc(nyx, pb, torch.zeros((160, 128), dtype=torch.uint16, device="cuda"), big)
    assert st == 6  # NYX_ERR_CAPACITY
    # the table recovers on the next call
    assert _noalloc(nyx, p, img, mask) == (0, 2)


def test_noalloc_error_paths(nyx):
    """Errors that the entry point reports without a result: a batch beyond
    its fixed limit (rejected before any launch), a negative label, and a
    mask with far more labels than the table holds, which must end with a
    capacity error after a short scan rather than a table probed slot by
    slot."""
    import time

    img = torch.zeros((64, 64), dtype=torch.uint16, device="cuda")
    mask = torch.zeros((64, 64), dtype=torch.int32, device="cuda")
    p = _params(nyx, (64, 64), 2, 0)
    p.batch = 1025  # one more image than NYX_NOALLOC_MAX_BATCH
    assert _noalloc(nyx, p, img, mask)[0] == 6  # NYX_ERR_CAPACITY
    p = _params(nyx, (64, 64), 2, 0)
    mask[3, 5] = -2
    assert _noalloc(nyx, p, img, mask)[0] == 4  # NYX_ERR_BAD_LABEL
    mask[3, 5] = 0
    assert _noalloc(nyx, p, img, mask) == (0, 0)
    # ~40K distinct labels, 2.5x the limit
    many = torch.arange(1, 256 * 160 + 1, dtype=torch.int32, device="cuda").reshape(256, 160)
    pm = _params(nyx, (256, 160), 2, 0)
    zeros = torch.zeros((256, 160), dtype=torch.uint16, device="cuda")
    _noalloc(nyx, pm, zeros, many)  # first call: module load and set-up
    t0 = time.perf_counter()
    st, _ = _noalloc(nyx, pm, zeros, many)
    assert st == 6
    assert time.perf_counter() - t0 < 1.0
    assert _noalloc(nyx, p, img, mask) == (0, 0)
