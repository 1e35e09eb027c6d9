"""Soft-feature planning (section "Feature Control and Tunability").

A soft feature's compute time is ordered by its hyperparameters: a larger
integer hyperparameter costs more (Eq. 2), and a superset of a set-valued
one costs more (Eq. 3), so the two together span a grid of ordered compute
times (Eqs. 4-5).  For the GLCM the integer hyperparameter is the grey depth
Ng and the set-valued one the set of distances.  `timing_grid` measures that
grid on the GPU path and `monotone_report` checks the ordering.

Which point of the grid to use for categorisation is chosen on a labelled
calibration set by a separability loss; Eq. 8 gives the class-unbiased ratio
of between- to within-class variance, implemented by `f_ratio` and swept over
the grid by `separability_grid`.

Host-side analysis only: every feature value comes from the CUDA path
through the Extractor; nothing here computes a feature.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

# Table S3 rows 140-174: the GLCM features the library computes
GLCM_FEATURES = ["ASM", "ACOR", "CLUPROM", "CLUSHADE", "CLUTEND", "CONTRAST", "CORR", "DIFAVE", "DIFENTRO", "DIFVAR",
                 "DIS", "ENERGY", "ENTROPY", "HOM1", "HOM2", "IDM", "INFOMEAS1", "INFOMEAS2", "IDMN", "ID", "IDN",
                 "IV", "JAVE", "JE", "JMAX", "SUMAVE", "SUMENT", "JVAR", "SUMVAR", "VARIANCE"]


def f_ratio(values: np.ndarray, classes: np.ndarray) -> float:
    """Eq. 8: (N - K) sum_i n_i (mean_i - mean)^2 / ((K - 1) sum_i sum_j
    (f_ij - mean_i)^2) over the samples with a finite value and a class
    >= 0.  NaN when fewer than two classes remain or the within-class sum
    is zero."""
    v = np.asarray(values, dtype=np.float64)
    c = np.asarray(classes)
    ok = np.isfinite(v) & (c >= 0)
    v, c = v[ok], c[ok]
    ks = np.unique(c)
    n, k = v.size, ks.size
    if k < 2 or n <= k:
        return float("nan")
    mean = v.mean()
    between = 0.0
    within = 0.0
    for cl in ks:
        x = v[c == cl]
        mi = x.mean()
        between += x.size * (mi - mean) ** 2
        within += float(np.sum((x - mi) ** 2))
    if within == 0.0:
        return float("nan")
    return (n - k) * between / ((k - 1) * within)


def monotone_report(t: np.ndarray, rel_tol: float = 0.0) -> Dict:
    """Check Eq. 5 on a grid t[k][j] (row k: the k-th distance set, nested
    supersets going down; column j: ascending grey depth): every step right
    and every step down must not be faster by more than rel_tol.  Returns
    the fraction of steps that hold and the violations."""
    t = np.asarray(t, dtype=np.float64)
    steps = 0
    bad: List[Tuple[str, int, int, float]] = []
    for k in range(t.shape[0]):
        for j in range(t.shape[1]):
            if j + 1 < t.shape[1]:
                steps += 1
                if t[k, j + 1] < t[k, j] * (1.0 - rel_tol):
                    bad.append(("levels", k, j, float(t[k, j + 1] / t[k, j])))
            if k + 1 < t.shape[0]:
                steps += 1
                if t[k + 1, j] < t[k, j] * (1.0 - rel_tol):
                    bad.append(("dists", k, j, float(t[k + 1, j] / t[k, j])))
    return {"steps": steps, "holds": steps - len(bad), "fraction": (steps - len(bad)) / max(steps, 1),
            "violations": bad}


def _extractor(w, levels: int, dists: Sequence[int], max_rois: int):
    import torch

    from . import nyx

    dt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
    return nyx.Extractor(w.image.shape, dt, ndim=w.ndim, glcm_levels=levels, dists=tuple(dists),
                         features=["GLCM_" + f for f in GLCM_FEATURES], max_rois=max_rois)


def timing_grid(w, levels: Sequence[int], dist_sets: Sequence[Sequence[int]], steps: int = 20, warmup: int = 3,
                max_rois: int = 8192) -> np.ndarray:
    """Median ms of a GLCM-only extraction (CUDA-graph replays, CUDA events)
    for every (distance set, grey depth) of the grid."""
    import torch

    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    out = np.zeros((len(dist_sets), len(levels)))
    for k, ds in enumerate(dist_sets):
        for j, ng in enumerate(levels):
            ex = _extractor(w, ng, ds, max_rois)
            table = torch.empty((max_rois, len(ex.columns)), dtype=torch.float64, device="cuda")
            for _ in range(warmup):
                ex.extract_into(img, mask, table)
            torch.cuda.synchronize()
            times = []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                ex.extract_into(img, mask, table)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ex.sync_status()
            out[k, j] = float(np.median(times))
    return out


def separability_grid(w, classes: np.ndarray, levels: Sequence[int], dist_sets: Sequence[Sequence[int]],
                      max_rois: int = 8192) -> Dict:
    """Eq. 8 for every GLCM feature (mean over directions at the first
    distance of the set) at every grid point.  classes[label] is the class
    of each label.  Returns the per-point best feature and its ratio, and the
    grid point that maximises each feature's ratio (the selection of Eq. 6
    on one calibration set)."""
    import torch

    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    ratio = {f: np.full((len(dist_sets), len(levels)), np.nan) for f in GLCM_FEATURES}
    for k, ds in enumerate(dist_sets):
        for j, ng in enumerate(levels):
            ex = _extractor(w, ng, ds, max_rois)
            tab = ex(img, mask).cpu().numpy()
            ex.sync_status()
            cols = {c: i for i, c in enumerate(ex.columns)}
            cl = classes[tab[:, cols["LABEL"]].astype(np.int64)]
            for f in GLCM_FEATURES:
                ratio[f][k, j] = f_ratio(tab[:, cols[f"GLCM_{f}_D{ds[0]}"]], cl)
    best_point = {}
    for f, r in ratio.items():
        if np.all(np.isnan(r)):
            continue
        k, j = np.unravel_index(np.nanargmax(r), r.shape)
        best_point[f] = {"dists": list(dist_sets[k]), "levels": int(levels[j]), "ratio": float(r[k, j])}
    best_feature = [[max(GLCM_FEATURES, key=lambda f: -np.inf if np.isnan(ratio[f][k, j]) else ratio[f][k, j])
                     for j in range(len(levels))] for k in range(len(dist_sets))]
    return {"ratio": {f: r.tolist() for f, r in ratio.items()}, "best_point": best_point,
            "best_feature": best_feature}
