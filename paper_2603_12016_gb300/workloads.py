"""Seeded synthetic image + label-mask workloads.

The paper measures on TissueNet (2D fluorescence), the Medical Segmentation
Decathlon (3D CT/MR) and a synthetic slide set of varying ROI size and count
(Fig. 3 and its "scalability" paragraph).  None of those datasets is
available here, so these generators produce inputs with the same shape of
problem: an intensity image plus an int32 label mask whose ROIs have the
size ranges and counts of the benchmark configurations.

This module holds no feature arithmetic: it only draws random numbers and
paints shapes.  Both the CUDA path and the CPU oracle receive its arrays.
Every generator is deterministic in its seed (NumPy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, Tuple

import numpy as np


@dataclass
class Workload:
    name: str
    image: np.ndarray          # [batch,] [z,] y, x
    mask: np.ndarray           # int32, same shape
    ndim: int                  # spatial dimensions (2 or 3)
    params: Dict = field(default_factory=dict)   # extraction hyperparameters
    meta: Dict = field(default_factory=dict)     # realised counts / sizes


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _relabel_drop_small(mask: np.ndarray, min_px: int) -> np.ndarray:
    """Remove labels with fewer than min_px pixels (set to background)."""
    labels, counts = np.unique(mask, return_counts=True)
    small = labels[(counts < min_px) & (labels > 0)]
    if len(small):
        mask[np.isin(mask, small)] = 0
    return mask


def _meta(mask: np.ndarray) -> Dict:
    labels, counts = np.unique(mask[mask > 0], return_counts=True)
    return {
        "n_roi": int(len(labels)),
        "roi_px_total": int(counts.sum()) if len(counts) else 0,
        "roi_px_min": int(counts.min()) if len(counts) else 0,
        "roi_px_max": int(counts.max()) if len(counts) else 0,
        "roi_px_median": float(np.median(counts)) if len(counts) else 0.0,
        "coverage": float(counts.sum() / mask.size) if len(counts) else 0.0,
    }


# ---------------------------------------------------------------------------
# 2D small: Gaussian blobs, Voronoi ROIs cut by a per-blob radius

def blobs_2d(size: int = 256, n_blobs: int = 64, seed: int = 1001, ng: int = 32) -> Workload:
    """256x256 uint16: Gamma(k=2, theta=300) background plus Gaussian blobs
    (sigma 3-10 px, peak 2000-40000).  The mask is the Voronoi partition of
    the blob centres, restricted to a disc per blob whose area is drawn from
    [50, 1500] px."""
    rng = _rng(seed)
    img = rng.gamma(2.0, 300.0, size=(size, size))
    cy = rng.uniform(8, size - 8, n_blobs)
    cx = rng.uniform(8, size - 8, n_blobs)
    sig = rng.uniform(3, 10, n_blobs)
    peak = rng.uniform(2000, 40000, n_blobs)
    area = rng.uniform(50, 1500, n_blobs)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    d2 = (yy[None] - cy[:, None, None]) ** 2 + (xx[None] - cx[:, None, None]) ** 2
    for k in range(n_blobs):
        img += peak[k] * np.exp(-d2[k] / (2 * sig[k] ** 2))
    owner = np.argmin(d2, axis=0)
    radius2 = area / math.pi
    mine = np.take_along_axis(d2, owner[None], 0)[0]
    mask = np.where(mine <= radius2[owner], owner + 1, 0).astype(np.int32)
    mask = _relabel_drop_small(mask, 20)
    img = np.clip(np.rint(img), 0, 65535).astype(np.uint16)
    return Workload("blobs2d_256_u16_64roi", img, mask, 2,
                    params=dict(glcm_levels=ng, dists=(1,), hist_bins=256), meta=_meta(mask))


# ---------------------------------------------------------------------------
# 2D fluorescence-like: ellipses on Gamma background with salt noise

def _paint_ellipses(mask, img, cy, cx, a, b, th, labels, value_fn):
    H, W = mask.shape
    for k in range(len(cy)):
        r = max(a[k], b[k]) + 1
        y0, y1 = max(0, int(cy[k] - r)), min(H, int(cy[k] + r) + 2)
        x0, x1 = max(0, int(cx[k] - r)), min(W, int(cx[k] + r) + 2)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        dy, dx = yy - cy[k], xx - cx[k]
        c, s = math.cos(th[k]), math.sin(th[k])
        u = (dx * c + dy * s) / a[k]
        v = (-dx * s + dy * c) / b[k]
        inside = u * u + v * v <= 1.0
        mask[y0:y1, x0:x1][inside] = labels[k]
        if img is not None:
            sub = img[y0:y1, x0:x1]
            sub[inside] = value_fn(k, int(inside.sum()), sub[inside])


def nuclei_2d(size: int = 2048, n_roi: int = 4000, seed: int = 1002, ng: int = 256,
              dists=(1, 2), salt: float = 0.02, axis_range=(4.0, 40.0), min_px: int = 50) -> Workload:
    """2048x2048 uint16 fluorescence-like image: Gamma(2, 300) background,
    n_roi ellipses (log-uniform semi-axes in axis_range, random angle) whose
    brightness ~ lognormal(mu=8, sigma=0.6) is added with +-20% per-pixel
    texture, then `salt` of all pixels set to 65535.  Ellipses are painted in
    random order (later ones overwrite); ROIs under min_px are dropped."""
    rng = _rng(seed)
    img = rng.gamma(2.0, 300.0, size=(size, size))
    mask = np.zeros((size, size), dtype=np.int32)
    lo, hi = math.log(axis_range[0]), math.log(axis_range[1])
    a = np.exp(rng.uniform(lo, hi, n_roi))
    b = np.exp(rng.uniform(lo, hi, n_roi))
    th = rng.uniform(0, math.pi, n_roi)
    cy = rng.uniform(0, size, n_roi)
    cx = rng.uniform(0, size, n_roi)
    bright = rng.lognormal(8.0, 0.6, n_roi)
    labels = rng.permutation(n_roi).astype(np.int32) + 1
    tex = rng.uniform(0.8, 1.2, size=(size, size))

    def val(k, n, cur):
        return cur + bright[k]

    _paint_ellipses(mask, img, cy, cx, a, b, th, labels, val)
    inroi = mask > 0
    img[inroi] = img[inroi] * tex[inroi]
    salt_px = rng.random((size, size)) < salt
    img[salt_px] = 65535
    mask = _relabel_drop_small(mask, min_px)
    img = np.clip(np.rint(img), 0, 65535).astype(np.uint16)
    return Workload(f"nuclei2d_{size}_u16_{n_roi}roi", img, mask, 2,
                    params=dict(glcm_levels=ng, dists=tuple(dists), hist_bins=256), meta=_meta(mask))


def texture_classes_2d(size: int = 1024, n_roi: int = 600, n_classes: int = 3, seed: int = 1006, ng: int = 64,
                       dists=(1,)) -> Workload:
    """Labelled texture classes for the separability ratio of Eq. 8: uint16
    ellipses (log-uniform semi-axes in [8, 24]) on a Gamma(2, 100)
    background.  Every ROI draws a class c in [0, n_classes) and a brightness
    ~ lognormal(mu=7.5, sigma=0.3) shared by all classes; its texture is
    Gaussian noise of 15% of the brightness smoothed with sigma = c (c = 0:
    unsmoothed), so the classes differ in texture coarseness, not in level.
    meta["classes"][label] is the class of each label (-1 for none)."""
    from scipy.ndimage import gaussian_filter

    rng = _rng(seed)
    img = rng.gamma(2.0, 100.0, size=(size, size))
    mask = np.zeros((size, size), dtype=np.int32)
    lo, hi = math.log(8.0), math.log(24.0)
    a = np.exp(rng.uniform(lo, hi, n_roi))
    b = np.exp(rng.uniform(lo, hi, n_roi))
    th = rng.uniform(0, math.pi, n_roi)
    cy = rng.uniform(0, size, n_roi)
    cx = rng.uniform(0, size, n_roi)
    bright = rng.lognormal(7.5, 0.3, n_roi)
    cls = rng.integers(0, n_classes, n_roi)
    labels = rng.permutation(n_roi).astype(np.int32) + 1
    fields = []
    for c in range(n_classes):
        f = rng.normal(size=(size, size))
        if c > 0:
            f = gaussian_filter(f, sigma=float(c))
            f /= f.std()
        fields.append(f)

    def val(k, n, cur):
        return cur * 0 + bright[k]

    _paint_ellipses(mask, img, cy, cx, a, b, th, labels, val)
    classes = np.full(n_roi + 1, -1, dtype=np.int64)
    classes[labels] = cls
    inroi = mask > 0
    cmap = classes[mask]
    for c in range(n_classes):
        sel = inroi & (cmap == c)
        img[sel] = img[sel] * (1.0 + 0.15 * fields[c][sel])
    mask = _relabel_drop_small(mask, 60)
    img = np.clip(np.rint(img), 0, 65535).astype(np.uint16)
    meta = _meta(mask)
    meta["classes"] = classes
    return Workload(f"textures2d_{size}_u16_{n_roi}roi_{n_classes}cls", img, mask, 2,
                    params=dict(glcm_levels=ng, dists=tuple(dists), hist_bins=256), meta=meta)


def scalability_2d(roi_px: int, n_roi: int, seed: int = 1007, ng: int = 64, dists=(1,)) -> Workload:
    """n_roi disks of about roi_px pixels each on a jittered square grid
    (cell side 1.5 diameters, so disks never touch), uint16: Gamma(2, 300)
    background, per-disk brightness ~ lognormal(mu=8, sigma=0.6) with +-20%
    per-pixel texture.  Image side = grid cells x cell side."""
    rng = _rng(seed)
    r = math.sqrt(roi_px / math.pi)
    cell = int(math.ceil(3.0 * r)) + 2
    g = int(math.ceil(math.sqrt(n_roi)))
    size = g * cell
    img = rng.gamma(2.0, 300.0, size=(size, size))
    mask = np.zeros((size, size), dtype=np.int32)
    slots = rng.permutation(g * g)[:n_roi]
    bright = rng.lognormal(8.0, 0.6, n_roi)
    span = max(cell - 2 * r - 2, 0.0)
    for k, sl in enumerate(slots):
        cy = (sl // g) * cell + r + 1 + rng.uniform(0, span)
        cx = (sl % g) * cell + r + 1 + rng.uniform(0, span)
        y0, y1 = max(0, int(cy - r) - 1), min(size, int(cy + r) + 2)
        x0, x1 = max(0, int(cx - r) - 1), min(size, int(cx + r) + 2)
        yy, xx = np.mgrid[y0:y1, x0:x1]
        inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r
        mask[y0:y1, x0:x1][inside] = k + 1
        img[y0:y1, x0:x1][inside] += bright[k]
    inroi = mask > 0
    img[inroi] *= rng.uniform(0.8, 1.2, size=int(inroi.sum()))
    img = np.clip(np.rint(img), 0, 65535).astype(np.uint16)
    return Workload(f"disks2d_{roi_px}px_x{n_roi}", img, mask, 2,
                    params=dict(glcm_levels=ng, dists=tuple(dists), hist_bins=256), meta=_meta(mask))


# ---------------------------------------------------------------------------
# 3D CT-like volume: smoothed random field + ellipsoids

def _smooth_field(rng, shape, sigma):
    from scipy.ndimage import gaussian_filter

    f = gaussian_filter(rng.standard_normal(shape).astype(np.float32), sigma=sigma, mode="wrap")
    f /= max(float(f.std()), 1e-6)
    return f


def ct_3d(shape=(128, 512, 512), n_roi: int = 200, seed: int = 1003, ng: int = 64,
          vol_range=(1e3, 1e6), force_extremes: bool = True) -> Workload:
    """512x512x128 int16 in [-1000, 3000]: a Gaussian-smoothed (sigma = 4 vox)
    random field (background around -300) plus n_roi ellipsoids with volumes
    log-uniform in vol_range (one forced to each end), each with a positive
    mean interior (200-1500 HU plus the field).  The volumes add up to most
    of the image, so ellipsoids are placed largest first, each at the best
    of up to 64 seeded candidate centres by the number of still unlabelled
    voxels it covers, and label only those: every ROI survives, the small
    ones whole."""
    rng = _rng(seed)
    Z, Y, X = shape
    field = _smooth_field(rng, shape, 4.0)
    img = -300.0 + 250.0 * field
    mask = np.zeros(shape, dtype=np.int32)
    vol = np.exp(rng.uniform(math.log(vol_range[0]), math.log(vol_range[1]), n_roi))
    if force_extremes and n_roi >= 2:
        vol[0], vol[1] = vol_range[1], vol_range[0]
    order = np.argsort(-vol, kind="stable")  # largest first
    level = rng.uniform(200, 1500, n_roi)
    labels = rng.permutation(n_roi).astype(np.int32) + 1
    zmax_semi = (Z - 2) / 2.0
    for k in order:
        r = (3 * vol[k] / (4 * math.pi)) ** (1 / 3)
        ez = rng.uniform(0.7, 1.0)
        ey = rng.uniform(0.8, 1.3)
        c = min(r * ez, zmax_semi)
        ab = vol[k] * 3 / (4 * math.pi) / c
        a = math.sqrt(ab * ey)
        b = ab / a
        best = None
        for _ in range(64):  # the candidate centre covering the most unlabelled voxels
            cz = rng.uniform(c, Z - c) if Z > 2 * c else Z / 2
            cy = rng.uniform(0, Y)
            cx = rng.uniform(0, X)
            z0, z1 = max(0, int(cz - c) - 1), min(Z, int(cz + c) + 2)
            y0, y1 = max(0, int(cy - b) - 1), min(Y, int(cy + b) + 2)
            x0, x1 = max(0, int(cx - a) - 1), min(X, int(cx + a) + 2)
            zz, yy, xx = np.ogrid[z0:z1, y0:y1, x0:x1]
            inside = ((zz - cz) / c) ** 2 + ((yy - cy) / b) ** 2 + ((xx - cx) / a) ** 2 <= 1.0
            free = inside & (mask[z0:z1, y0:y1, x0:x1] == 0)
            nfree = int(free.sum())
            if best is None or nfree > best[0]:
                best = (nfree, (z0, z1, y0, y1, x0, x1), free)
            if nfree >= 0.99 * int(inside.sum()):
                break
        _, (z0, z1, y0, y1, x0, x1), free = best
        mask[z0:z1, y0:y1, x0:x1][free] = labels[k]
        sub = img[z0:z1, y0:y1, x0:x1]
        sub[free] = level[k] + 200.0 * field[z0:z1, y0:y1, x0:x1][free]
    mask = _relabel_drop_small(mask, 100)
    img = np.clip(np.rint(img), -1000, 3000).astype(np.int16)
    return Workload(f"ct3d_{X}x{Y}x{Z}_i16_{n_roi}roi", img, mask, 3,
                    params=dict(glcm_levels=ng, dists=(1,), hist_bins=256), meta=_meta(mask))


# ---------------------------------------------------------------------------
# batch of float32 blob images (differentiation workload)

def blob_batch_f32(batch: int = 64, size: int = 512, seed: int = 1004, roi_range=(4, 256),
                   px_range=(30, 20000), coverage: float = 0.7) -> Workload:
    """batch x size x size float32 images of Gaussian blobs on N(100, 10)
    background; image b holds n_b ROIs (log-uniform in roi_range) whose disc
    areas are log-uniform in px_range, scaled down so that the summed area
    stays under `coverage` of the image."""
    rng = _rng(seed)
    img = rng.normal(100.0, 10.0, size=(batch, size, size)).astype(np.float32)
    mask = np.zeros((batch, size, size), dtype=np.int32)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float32)
    lo, hi = math.log(roi_range[0]), math.log(roi_range[1])
    for bi in range(batch):
        n = int(round(math.exp(rng.uniform(lo, hi))))
        areas = np.exp(rng.uniform(math.log(px_range[0]), math.log(px_range[1]), n))
        tot = areas.sum()
        if tot > coverage * size * size:
            areas *= coverage * size * size / tot
        labels = rng.permutation(n).astype(np.int32) + 1
        for k in range(n):
            r = math.sqrt(max(areas[k], px_range[0]) / math.pi)
            cy, cx = rng.uniform(r, size - r), rng.uniform(r, size - r)
            amp = rng.uniform(200, 2000)
            sig = max(r / 2.0, 1.0)
            y0, y1 = max(0, int(cy - r) - 1), min(size, int(cy + r) + 2)
            x0, x1 = max(0, int(cx - r) - 1), min(size, int(cx + r) + 2)
            d2 = (yy[y0:y1, x0:x1] - cy) ** 2 + (xx[y0:y1, x0:x1] - cx) ** 2
            img[bi, y0:y1, x0:x1] += (amp * np.exp(-d2 / (2 * sig * sig))).astype(np.float32)
            mask[bi, y0:y1, x0:x1][d2 <= r * r] = labels[k]
    for bi in range(batch):
        mask[bi] = _relabel_drop_small(mask[bi], 10)
    return Workload(f"blobbatch_{batch}x{size}_f32", img, mask, 2,
                    params=dict(glcm_levels=0, dists=(1,), hist_bins=256), meta=_meta(mask))


# ---------------------------------------------------------------------------
# streamed mosaic: generated tile by tile from one global ROI placement

@dataclass
class Mosaic:
    """A size x size uint16 mosaic produced tile by tile.  tile(x0, y0, w, h)
    returns (image, mask) of that window; windows agree where they overlap,
    so ROIs crossing tile borders are consistent."""
    name: str
    size: int
    tile_size: int
    n_roi: int
    params: Dict
    _cy: np.ndarray = field(repr=False, default=None)
    _cx: np.ndarray = field(repr=False, default=None)
    _a: np.ndarray = field(repr=False, default=None)
    _b: np.ndarray = field(repr=False, default=None)
    _th: np.ndarray = field(repr=False, default=None)
    _bright: np.ndarray = field(repr=False, default=None)
    _labels: np.ndarray = field(repr=False, default=None)
    _order: np.ndarray = field(repr=False, default=None)
    _seed: int = 0
    _kw: Dict = field(repr=False, default=None)  # mosaic_2d arguments (rebuilds it in worker processes)

    def tile(self, x0: int, y0: int, w: int, h: int):
        # background and texture depend on the pixel position only (a hash of
        # (seed, y, x)), so overlapping windows agree
        yy, xx = np.mgrid[y0:y0 + h, x0:x0 + w].astype(np.uint64)
        hsh = (yy * np.uint64(0x9E3779B97F4A7C15) ^ xx * np.uint64(0xC2B2AE3D27D4EB4F) ^
               np.uint64(self._seed * 0x165667B19E3779F9 % (1 << 63)))
        hsh ^= hsh >> np.uint64(29)
        hsh *= np.uint64(0xBF58476D1CE4E5B9)
        hsh ^= hsh >> np.uint64(32)
        u1 = ((hsh & np.uint64(0xFFFFFF)).astype(np.float64) + 0.5) / float(1 << 24)
        u2 = (((hsh >> np.uint64(24)) & np.uint64(0xFFFFFF)).astype(np.float64) + 0.5) / float(1 << 24)
        img = -300.0 * np.log(u1 * u2)          # Gamma(2, 300): sum of two exponentials
        mask = np.zeros((h, w), dtype=np.int32)
        # ellipses touching the window, painted in the global order
        r = np.maximum(self._a, self._b)
        hit = np.flatnonzero((self._cy + r >= y0) & (self._cy - r < y0 + h) &
                             (self._cx + r >= x0) & (self._cx - r < x0 + w))
        hit = hit[np.argsort(self._order[hit], kind="stable")]
        for k in hit:
            ry0, ry1 = max(y0, int(self._cy[k] - r[k]) - 1), min(y0 + h, int(self._cy[k] + r[k]) + 2)
            rx0, rx1 = max(x0, int(self._cx[k] - r[k]) - 1), min(x0 + w, int(self._cx[k] + r[k]) + 2)
            if ry1 <= ry0 or rx1 <= rx0:
                continue
            gy, gx = np.mgrid[ry0:ry1, rx0:rx1].astype(np.float64)
            dy, dx = gy - self._cy[k], gx - self._cx[k]
            c, s_ = math.cos(self._th[k]), math.sin(self._th[k])
            u = (dx * c + dy * s_) / self._a[k]
            v = (-dx * s_ + dy * c) / self._b[k]
            inside = u * u + v * v <= 1.0
            sub = mask[ry0 - y0:ry1 - y0, rx0 - x0:rx1 - x0]
            sub[inside] = self._labels[k]
            isub = img[ry0 - y0:ry1 - y0, rx0 - x0:rx1 - x0]
            isub[inside] = isub[inside] + self._bright[k]
        salt = u1 < 0.01
        img[salt] = 65535
        return np.clip(np.rint(img), 0, 65535).astype(np.uint16), mask

    def assemble(self, procs: int = 1):
        """The whole mosaic.  With procs > 1 the tiles are generated in that
        many processes (started with spawn, so call it before any CUDA use)."""
        img = np.empty((self.size, self.size), dtype=np.uint16)
        mask = np.empty((self.size, self.size), dtype=np.int32)
        t = self.tile_size
        jobs = [(x0, y0, min(t, self.size - x0), min(t, self.size - y0))
                for y0 in range(0, self.size, t) for x0 in range(0, self.size, t)]
        if procs > 1 and len(jobs) > 1:
            import multiprocessing as mp

            with mp.get_context("spawn").Pool(procs, initializer=_mosaic_worker_init, initargs=(self._kw,)) as pool:
                tiles = pool.imap(_mosaic_worker_tile, jobs)
                for (x0, y0, w, h), (ti, tm) in zip(jobs, tiles):
                    img[y0:y0 + h, x0:x0 + w], mask[y0:y0 + h, x0:x0 + w] = ti, tm
        else:
            for x0, y0, w, h in jobs:
                img[y0:y0 + h, x0:x0 + w], mask[y0:y0 + h, x0:x0 + w] = self.tile(x0, y0, w, h)
        return img, mask


_MOSAIC_WORKER = None


def _mosaic_worker_init(kw):
    global _MOSAIC_WORKER
    _MOSAIC_WORKER = mosaic_2d(**kw)


def _mosaic_worker_tile(job):
    return _MOSAIC_WORKER.tile(*job)


def mosaic_2d(size: int = 32768, tile: int = 4096, n_roi: int = 500_000, seed: int = 1005, ng: int = 64,
              area_range=(20.0, 1e4)) -> Mosaic:
    """size x size uint16 mosaic (whole-slide stand-in): Gamma(2, 300)
    background, 1% salt, n_roi ellipses placed once over the whole mosaic
    (areas log-uniform in area_range, aspect 1-2, random angle, lognormal
    brightness), painted in a random global order so that later ones
    overwrite earlier ones; many cross tile borders."""
    rng = _rng(seed)
    area = np.exp(rng.uniform(math.log(area_range[0]), math.log(area_range[1]), n_roi))
    asp = rng.uniform(1.0, 2.0, n_roi)
    b = np.sqrt(area / (math.pi * asp))
    a = b * asp
    kw = dict(size=size, tile=tile, n_roi=n_roi, seed=seed, ng=ng, area_range=area_range)
    return Mosaic(name=f"mosaic_{size}_u16_{n_roi}roi", size=size, tile_size=tile, n_roi=n_roi, _kw=kw,
                  params=dict(glcm_levels=ng, dists=(1,), hist_bins=256),
                  _cy=rng.uniform(0, size, n_roi), _cx=rng.uniform(0, size, n_roi), _a=a, _b=b,
                  _th=rng.uniform(0, math.pi, n_roi), _bright=rng.lognormal(8.0, 0.6, n_roi),
                  _labels=rng.permutation(n_roi).astype(np.int32) + 1, _order=rng.permutation(n_roi), _seed=seed)


# ---------------------------------------------------------------------------
# named configurations (sizes of the benchmark table) and small variants

def mosaic_workload(name: str, seed_offset: int = 0, procs: int = 1) -> Workload:
    """The streamed mosaic as one assembled workload: "mosaic" (32768^2, 4096^2
    tiles, 500,000 placed ROIs) or "mosaic_small" (8192^2, 1024^2 tiles,
    32,000)."""
    big = name == "mosaic"
    m = mosaic_2d(size=32768 if big else 8192, tile=4096 if big else 1024, n_roi=500_000 if big else 32_000,
                  seed=1005 + seed_offset)
    img, mask = m.assemble(procs)
    n_roi = int(np.count_nonzero(np.bincount(mask.ravel())[1:]))
    return Workload(m.name, img, mask, 2, params=dict(m.params), meta={"n_roi": n_roi, "tile": m.tile_size})


def config(name: str, seed_offset: int = 0) -> Workload:
    if name.startswith("mosaic"):
        return mosaic_workload(name, seed_offset)
    if name == "blobs2d":
        return blobs_2d(seed=1001 + seed_offset)
    if name == "nuclei2d":
        return nuclei_2d(seed=1002 + seed_offset)
    if name == "nuclei2d_small":
        return nuclei_2d(size=512, n_roi=250, seed=1102 + seed_offset)
    if name == "ct3d":
        return ct_3d(seed=1003 + seed_offset)
    if name == "ct3d_small":
        return ct_3d(shape=(32, 96, 96), n_roi=12, seed=1103 + seed_offset, vol_range=(200, 2e4))
    if name == "blobbatch":
        return blob_batch_f32(seed=1004 + seed_offset)
    if name == "blobbatch_small":
        return blob_batch_f32(batch=4, size=128, seed=1104 + seed_offset, roi_range=(4, 32), px_range=(30, 2000))
    raise KeyError(name)
