"""Backward pass of the smooth intensity features on the GPU (nyx_backward
through the C ABI, and FeatureLayer through autograd) against the oracle's
analytic FP64 gradient and against central finite differences (h = 1e-3) of
the FP64 oracle forward on sampled pixels; tolerance rel 1e-3."""
import numpy as np
import pytest

import oracle
from paper_2603_12016_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SMOOTH = ["MEAN", "VARIANCE", "VARIANCE_BIASED", "STDDEV", "STDDEV_BIASED", "SKEWNESS", "KURTOSIS", "EXCESS_KURTOSIS",
          "HYPERSKEWNESS", "HYPERFLATNESS", "ENERGY", "ROOT_MEAN_SQUARED", "STANDARD_ERROR", "MEAN_ABSOLUTE_DEVIATION",
          "INTEGRATED_INTENSITY", "WEIGHTED_CENTROID_X", "WEIGHTED_CENTROID_Y", "WEIGHTED_CENTROID_Z",
          "MASS_DISPLACEMENT", "COV", "EDGE_INTEGRATED_INTENSITY", "EDGE_MEAN_INTENSITY", "EDGE_STDDEV_INTENSITY"]
FAMILIES = ["INT_M", "INT_MU", "INT_ETA", "INT_NU", "INT_HU"]
RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12016_gb300 import build

    build.build()


def _upstream(cols, table, rng):
    """Random dL/dF scaled by 1/|F| per column (first-order central moments,
    identically zero, get no gradient)."""
    g = np.zeros_like(table)
    for j, c in enumerate(cols):
        if c in ("LABEL", "IMAGE", "AREA") or c.startswith("BBOX") or c.startswith("CENTROID"):
            continue
        if c in ("INT_MU10", "INT_MU01", "INT_MU100", "INT_MU010", "INT_MU001"):
            continue
        col = table[:, j]
        scale = np.where(np.isfinite(col), np.abs(col), 1.0) + 1e-3
        g[:, j] = rng.normal(size=len(col)) / scale
    return g


def _check(w, ndim, n_fd=24):
    from paper_2603_12016_gb300 import nyx

    rng = np.random.default_rng(11)
    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    layer = nyx.FeatureLayer(w.image.shape, ndim=ndim, max_rois=4096, features=SMOOTH + FAMILIES)
    x = img.clone().requires_grad_(True)
    table = layer(x, mask)
    cols = layer.columns
    tab = table.detach().cpu().numpy()
    g = _upstream(cols, tab, rng)
    table.backward(torch.from_numpy(g).cuda())
    got = x.grad.detach().cpu().numpy().astype(np.float64)
    gtab = {c: g[:, j] for j, c in enumerate(cols)}
    ref = oracle.grad(w.image.astype(np.float64), w.mask, ndim, gtab)
    inroi = w.mask > 0
    assert np.all(got[~inroi] == 0)
    # per-ROI scale: the largest reference gradient magnitude in that ROI
    labels = w.mask.astype(np.int64)
    if labels.ndim == 3 and ndim == 2:
        bidx = np.broadcast_to(np.arange(labels.shape[0], dtype=np.int64)[:, None, None], labels.shape)
    else:
        bidx = np.zeros_like(labels)
    keyarr = (bidx << 32) + labels
    worst = 0.0
    for k in np.unique(keyarr[labels > 0]):
        sel = keyarr == k
        r = ref[sel]
        err = np.max(np.abs(got[sel] - r)) / (np.max(np.abs(r)) + 1e-30)
        worst = max(worst, err)
        assert err <= RTOL, (k >> 32, k & 0xFFFFFFFF, err)
    # finite differences of the FP64 oracle forward on sampled ROI pixels
    names = [c for c in cols if np.any(gtab[c] != 0)]
    img64 = w.image.astype(np.float64)

    def loss(im):
        t = oracle.extract(im, w.mask, ndim, ng=0)
        return sum(float(np.sum(gtab[c] * t[c])) for c in names)

    idx = rng.choice(np.flatnonzero(inroi.ravel()), size=n_fd, replace=False)
    for i in idx:
        ip, im_ = img64.copy(), img64.copy()
        ip.flat[i] += 1e-3
        im_.flat[i] -= 1e-3
        fd = (loss(ip) - loss(im_)) / 2e-3
        assert abs(got.flat[i] - fd) <= RTOL * max(abs(fd), 1e-3 * np.max(np.abs(ref))), (i, got.flat[i], fd)
    return worst


def test_backward_blob_batch_f32():
    w = W.config("blobbatch_small")
    _check(w, 2)


def test_backward_3d_volume_f32():
    v = W.ct_3d(shape=(16, 40, 40), n_roi=5, seed=99, vol_range=(150, 2000))
    w = W.Workload("ct_small_f32", v.image.astype(np.float32), v.mask, 3, params=v.params, meta=v.meta)
    _check(w, 3, n_fd=12)


def test_backward_requires_saved_forward():
    from paper_2603_12016_gb300 import nyx

    ex = nyx.Extractor((16, 16), torch.float32, glcm_levels=0, max_rois=64)
    img = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    mask = torch.ones((16, 16), dtype=torch.int32, device="cuda")
    ex(img, mask)  # forward without save_for_backward
    with pytest.raises(nyx.NyxError) as e:
        ex.backward(img, mask, torch.zeros((64, len(ex.columns)), dtype=torch.float64, device="cuda"))
    assert e.value.status == 10


def test_backward_big_rois_f32():
    """ROIs above 8192 px take the multi-block path; their saved state feeds
    the same backward kernels."""
    w = W.blob_batch_f32(batch=2, size=256, seed=2305, roi_range=(3, 5), px_range=(9000, 20000))
    assert np.bincount(w.mask.ravel())[1:].max() > 8192
    _check(w, 2, n_fd=8)


def test_backward_label_map_kept_or_rebuilt():
    """The forward pass saved for backward keeps its label -> ROI map: a
    backward on the same buffers reuses it, one on copies of them (or after
    another call released it) rebuilds it; all three give the same gradient."""
    from paper_2603_12016_gb300 import nyx

    w = W.config("blobbatch_small")
    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    ex = nyx.Extractor(w.image.shape, torch.float32, glcm_levels=0, max_rois=1024, features=SMOOTH + FAMILIES)
    table = ex(img, mask, save_for_backward=True)
    g = torch.randn(table.shape, dtype=torch.float64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    g_same = ex.backward(img, mask, g)                       # kept map
    ex(img, mask, save_for_backward=True)
    g_copy = ex.backward(img.clone(), mask.clone(), g)       # other buffers: rebuilt map
    ex(img, mask, save_for_backward=True)
    assert ex.count_rois(img, mask) == table.shape[0]        # releases the kept map
    g_after = ex.backward(img, mask, g)
    torch.cuda.synchronize()
    assert torch.equal(g_same, g_copy) and torch.equal(g_same, g_after)
    assert torch.count_nonzero(g_same[mask == 0]) == 0 and torch.count_nonzero(g_same) > 0


def test_backward_full_size_batch_sampled_fd():
    """The full differentiation workload (64 float32 512 x 512 images, ~3,000
    ROIs, sizes 30-20,000 px, the multi-block class included) in the launch
    configuration the benchmark times.  For a sample of ROIs: every pixel's
    GPU gradient against the oracle's analytic FP64 gradient, pixel by pixel
    at rel 1e-3 (floor: 1e-6 of the ROI's largest gradient, for pixels where
    the gradient crosses zero); and 32 random pixels per ROI against central
    finite differences (h = 1e-3) of the FP64 oracle forward, at rel 1e-3
    plus the difference quotient's own rounding noise.  That noise is
    measured, not assumed: |L(+h) + L(-h) - 2 L(0)| / (2h) for the same
    pixel, which is the rounding of the three loss evaluations (the
    curvature term is ~h L''/2, far below it).  Large features with small
    per-pixel derivatives (mu20 near the centroid of a 20,000 px ROI: 1.4e10
    against a change of 1e-2) make it reach 1e-2 of a pixel's gradient there.
    A ROI's features depend only on its own pixels and on its neighbours'
    labels (edge pixels), so both references are computed on a crop of the
    ROI's bounding box with a one-pixel margin."""
    from paper_2603_12016_gb300 import nyx

    w = W.config("blobbatch")
    rng = np.random.default_rng(29)
    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    n_roi = int(sum(len(np.unique(m[m > 0])) for m in w.mask))
    layer = nyx.FeatureLayer(w.image.shape, ndim=2, max_rois=8192, features=SMOOTH + FAMILIES)
    x = img.clone().requires_grad_(True)
    table = layer(x, mask)
    assert table.shape[0] == n_roi
    cols = layer.columns
    tab = table.detach().cpu().numpy()
    g = _upstream(cols, tab, rng)
    table.backward(torch.from_numpy(g).cuda())
    got = x.grad.detach().cpu().numpy().astype(np.float64)
    rows = [(int(b), int(l)) for b, l in zip(tab[:, cols.index("IMAGE")], tab[:, cols.index("LABEL")])]
    area = tab[:, cols.index("AREA")]
    pick = set(rng.choice(len(rows), size=10, replace=False).tolist()) | {int(np.argmax(area)), int(np.argmin(area))}
    assert area.max() > 8192  # the multi-block class is in the sample
    for r in sorted(pick):
        b, lab = rows[r]
        m = w.mask[b]
        ys, xs = np.nonzero(m == lab)
        y0, y1 = max(ys.min() - 1, 0), min(ys.max() + 2, m.shape[0])
        x0, x1 = max(xs.min() - 1, 0), min(xs.max() + 2, m.shape[1])
        cm = np.where(m[y0:y1, x0:x1] == lab, lab, 0).astype(np.int32)
        ci = w.image[b, y0:y1, x0:x1].astype(np.float64)
        names = [c for j, c in enumerate(cols) if g[r, j] != 0]
        gr = {c: g[r, cols.index(c)] for c in names}
        # analytic FP64 gradient, every pixel of the ROI
        ref = oracle.grad(ci, cm, 2, {c: np.array([v]) for c, v in gr.items()})
        gg = got[b, y0:y1, x0:x1]
        inr = cm > 0
        scale = np.max(np.abs(ref[inr]))
        bad = np.abs(gg[inr] - ref[inr]) > RTOL * np.maximum(np.abs(ref[inr]), 1e-3 * scale)
        assert not bad.any(), (b, lab, int(area[r]), gg[inr][bad][:4], ref[inr][bad][:4])

        def loss(im):
            t = oracle.extract(im, cm, 2, ng=0)
            return sum(gr[c] * float(t[c][0]) for c in names)

        l0 = loss(ci)
        for k in rng.choice(len(ys), size=min(32, len(ys)), replace=False):
            yy, xx = ys[k] - y0, xs[k] - x0
            ip, im_ = ci.copy(), ci.copy()
            ip[yy, xx] += 1e-3
            im_[yy, xx] -= 1e-3
            lp, lm = loss(ip), loss(im_)
            fd = (lp - lm) / 2e-3
            noise = abs(lp + lm - 2 * l0) / 2e-3
            gv = got[b, ys[k], xs[k]]
            assert abs(gv - fd) <= RTOL * abs(fd) + 4 * noise + 1e-6 * scale, (b, lab, int(area[r]), gv, fd, noise)
