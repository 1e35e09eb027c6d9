"""Helpers for GPU-vs-oracle parity tests.

Tolerances (stated by the build target; natural scales per feature so that
values that are zero by symmetry are compared against their scale):
  exact     : counts, bounding boxes, min/max/range, labels, order statistics
              (same FP64 operations on the same sorted values), mode value
  RTOL_STAT : 1e-5 for first-order statistics and moments
  RTOL_GLCM : 1e-4 for GLCM features (floors in glcm_scale)
  NGTDM / GLDM features: RTOL_STAT, relative, the GLDM variances on the
              unit scale of an integer dependence / grey level
|gpu - oracle| <= rtol * max(|oracle|, scale).
"""
from __future__ import annotations

import math
import re
from typing import Dict, List, Optional, Tuple

import numpy as np

RTOL_STAT = 1e-5
RTOL_GLCM = 1e-4

EXACT = {"LABEL", "IMAGE", "AREA", "BBOX_XMIN", "BBOX_YMIN", "BBOX_ZMIN", "BBOX_WIDTH", "BBOX_HEIGHT", "BBOX_DEPTH",
         "MIN", "MAX", "RANGE", "MEDIAN", "P01", "P10", "P25", "P75", "P90", "P99", "INTERQUARTILE_RANGE", "MODE",
         "EDGE_MIN_INTENSITY", "EDGE_MAX_INTENSITY"}
DIMENSIONLESS = {"MODE_PROBABILITY", "SKEWNESS", "KURTOSIS", "EXCESS_KURTOSIS", "HYPERSKEWNESS", "HYPERFLATNESS", "ENTROPY",
                 "UNIFORMITY", "COV", "QCOD", "COVERED_IMAGE_INTENSITY_RANGE", "UNIFORMITY_PIU"}


def moment_exps(name: str) -> Tuple[int, ...]:
    digits = "".join(ch for ch in name if ch.isdigit())
    return tuple(int(c) for c in digits)


def scales(t: Dict[str, np.ndarray], name: str, ndim: int) -> np.ndarray:
    """Natural scale of feature `name` for every ROI of oracle table t."""
    n = len(t["LABEL"])
    one = np.ones(n)
    std = np.sqrt(np.abs(t.get("VARIANCE_BIASED", one)))
    amax = np.maximum(np.abs(t.get("MIN", one)), np.abs(t.get("MAX", one)))
    ext = [t["BBOX_WIDTH"], t["BBOX_HEIGHT"], t.get("BBOX_DEPTH", one)]
    if name.startswith("GLCM_"):
        return glcm_scale(t, name)
    if name.startswith("GLDM_"):
        # dependences and grey levels are integers >= 1: their variances
        # (near zero when every pixel shares one value) on that unit scale
        if name in ("GLDM_DV", "GLDM_GLV"):
            return one
        return np.full(n, TINY)
    if name.startswith(("GLRLM_", "GLSZM_")):
        # the level and size variances vanish for one item or equal items,
        # the entropies for one (level, size) cell: unit scale; the rest are
        # positive means and ratios of positive sums
        if name.endswith(("_GLV", "_RV", "_ZV", "_RE", "_ZE")):
            return one
        return np.full(n, TINY)
    if name.startswith("NGTDM_"):
        # contrast, busyness, complexity and strength are exactly 0 in their
        # degenerate cases (one grey level, no neighbour differences)
        return np.full(n, TINY)
    if name in DIMENSIONLESS:
        return one
    if name in ("MEAN", "ROBUST_MEAN", "MEDIAN", "EDGE_MEAN_INTENSITY"):
        return np.maximum(std, amax * 1e-3)
    if name in ("MEAN_ABSOLUTE_DEVIATION", "MEDIAN_ABSOLUTE_DEVIATION", "ROBUST_MEAN_ABSOLUTE_DEVIATION",
                "STDDEV", "STDDEV_BIASED", "STANDARD_ERROR", "EDGE_STDDEV_INTENSITY"):
        return np.maximum(std, amax * 1e-3)
    if name in ("VARIANCE", "VARIANCE_BIASED"):
        return np.maximum(std ** 2, (amax * 1e-3) ** 2)
    if name.startswith("WEIGHTED_CENTROID") or name.startswith("CENTROID") or name == "MASS_DISPLACEMENT":
        return np.maximum(ext[0], ext[1])
    if name == "EDGE_INTEGRATED_INTENSITY":
        return np.abs(t["AREA"]) * amax
    if name in ("ENERGY", "ROOT_MEAN_SQUARED", "INTEGRATED_INTENSITY"):
        return np.abs(t["AREA"]) * amax ** (2 if name == "ENERGY" else 1) * (1 if name != "ROOT_MEAN_SQUARED" else
                                                                               1 / np.maximum(t["AREA"], 1))
    for pre in ("INT_", "BIN_"):
        if not name.startswith(pre):
            continue
        fam = name[len(pre):].rstrip("0123456789")
        e = moment_exps(name[len(pre) + len(fam):]) if fam != "HU" else ()
        w0 = (t["AREA"] * amax) if pre == "INT_" else t["AREA"].astype(float)
        mu00 = np.abs(t[pre + ("MU000" if ndim == 3 else "MU00")])
        mu00 = np.where(mu00 > 0, mu00, w0)
        if ndim == 2:
            sig = [np.sqrt(np.abs(t[pre + "MU20"]) / mu00), np.sqrt(np.abs(t[pre + "MU02"]) / mu00)]
        else:
            sig = [np.sqrt(np.abs(t[pre + "MU200"]) / mu00), np.sqrt(np.abs(t[pre + "MU020"]) / mu00),
                   np.sqrt(np.abs(t[pre + "MU002"]) / mu00)]
        sig = [np.maximum(s, 0.5) for s in sig]
        if fam == "MU":
            s = w0.copy()
            for a, k in enumerate(e):
                s = s * sig[a] ** k
            return s
        if fam == "M":
            s = w0.copy()
            for a, k in enumerate(e):
                s = s * np.maximum(ext[a], 1.0) ** k
            return s
        if fam == "ETA":
            o = sum(e)
            s = w0.copy()
            for a, k in enumerate(e):
                s = s * sig[a] ** k
            return s / mu00 ** (1 + o / (3 if ndim == 3 else 2))
        if fam == "NU":
            o = sum(e)
            s = w0.copy()
            for a, k in enumerate(e):
                s = s * np.maximum(ext[a], 1.0) ** k
            return s / mu00 ** (1 + o / 2)
        if fam == "HU":
            h = int(name[len(pre) + 2:])
            s2 = (sig[0] ** 2 + sig[1] ** 2) * w0 / mu00 ** 2
            deg = {1: 1, 2: 2, 3: 3, 4: 3, 5: 6, 6: 4, 7: 6}[h]
            return s2 ** deg
    return np.maximum(np.abs(t.get(name, one)), 1.0)


TINY = 1e-300


def glcm_scale(t: Dict[str, np.ndarray], name: str) -> np.ndarray:
    """Natural scale of a GLCM feature column (direction mean or per offset).
    Relative 1e-4 everywhere, with a floor only for features that vanish by
    symmetry or degeneracy, at the feature's own scale:
      CLUSHADE (zero for a symmetric sum distribution): CLUPROM^(3/4), the
        bound of sum |i + j - 2 mu|^3 p by Hoelder's inequality;
      CORR, INFOMEAS1, INFOMEAS2 (zero for uncorrelated / independent
        matrices; dimensionless, |value| <= 1): 1e-2;
      the entropies JE, ENTROPY, SUMENT, DIFENTRO (zero for a one-cell
        distribution): 1e-2 bit;
      CONTRAST, DIS, DIFAVE, DIFVAR, IV (zero when every pair lies on the
        diagonal): their squared / first level unit times 1e-12;
      the central moments CLUTEND, SUMVAR, CLUPROM, JVAR, VARIANCE (zero for
        one grey level): 1e-10 times the matching power of the mean level,
        the size of the FP64 cancellation in the oracle's two-pass form;
      everything else (ASM, ENERGY, JMAX, ACOR, JAVE, SUMAVE, the inverse
        differences): strictly positive, relative only."""
    n = len(t["LABEL"])
    base = name[len("GLCM_"):]
    m = re.match(r"([A-Z0-9]+?)(_D\d+(?:_A\d+|_O\d+)?)$", base)
    feat, suf = (m.group(1), m.group(2)) if m else (base, "")

    def col(f):
        v = t.get("GLCM_" + f + suf)
        return np.abs(v) if v is not None else np.ones(n)

    if feat == "CLUSHADE":
        return col("CLUPROM") ** 0.75
    if feat in ("CORR", "INFOMEAS1", "INFOMEAS2", "JE", "ENTROPY", "SUMENT", "DIFENTRO"):
        return np.full(n, 1e-2)
    if feat in ("CONTRAST", "DIS", "DIFAVE", "DIFVAR", "IV"):
        return np.full(n, 1e-12)
    if feat in ("CLUTEND", "SUMVAR"):
        return 1e-10 * col("SUMAVE") ** 2
    if feat == "CLUPROM":
        return 1e-10 * col("SUMAVE") ** 4
    if feat in ("JVAR", "VARIANCE"):
        return 1e-10 * col("JAVE") ** 2
    return np.full(n, TINY)


def compare(gpu: Dict[str, np.ndarray], orc: Dict[str, np.ndarray], ndim: int, rtol_stat=RTOL_STAT,
            rtol_glcm=RTOL_GLCM, skip=()) -> List[str]:
    """Return a list of failure descriptions (empty = parity)."""
    fails = []
    assert np.array_equal(gpu["LABEL"], orc["LABEL"]) and np.array_equal(gpu["IMAGE"], orc["IMAGE"]), \
        "ROI sets differ"
    for name, g in gpu.items():
        if name in skip or name not in orc:
            continue
        o = orc[name]
        both_nan = np.isnan(g) & np.isnan(o)
        if name in EXACT:
            bad = ~(both_nan | (g == o))
            if bad.any():
                i = int(np.flatnonzero(bad)[0])
                fails.append(f"{name}: not bit-exact at row {i}: gpu {g[i]!r} oracle {o[i]!r} ({bad.sum()} rows)")
            continue
        rtol = rtol_glcm if name.startswith("GLCM_") else rtol_stat
        sc = scales(orc, name, ndim)
        tol = rtol * np.maximum(np.abs(o), sc)
        with np.errstate(invalid="ignore"):
            bad = ~(both_nan | (np.abs(g - o) <= tol))
        if bad.any():
            i = int(np.flatnonzero(bad)[np.argmax((np.abs(g - o) / tol)[bad])])
            fails.append(f"{name}: row {i} gpu {g[i]!r} oracle {o[i]!r} tol {tol[i]:.3g} ({bad.sum()}/{len(g)} rows)")
    return fails


def gpu_table(ex, img_t, mask_t) -> Dict[str, np.ndarray]:
    table = ex(img_t, mask_t).cpu().numpy()
    return {c: table[:, i] for i, c in enumerate(ex.columns)}


def to_torch(a: np.ndarray, device="cuda"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(device)
