"""Scalability over ROI size and ROI count on the GPU path (the study of
Fig. 3f/g): device time of an extraction already resident in HBM, end-to-end
time through the public call with host buffers (pinned host -> device copies
of image and mask, the extraction, the table back to the host), and the cost
of each feature group on one image.

GPU measurement only; every feature is computed by the CUDA path.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

GLCM = ["GLCM_" + f for f in ("ASM", "ACOR", "CLUPROM", "CLUSHADE", "CLUTEND", "CONTRAST", "CORR", "DIFAVE", "DIFENTRO",
                                "DIFVAR", "DIS", "ENERGY", "ENTROPY", "HOM1", "HOM2", "IDM", "INFOMEAS1", "INFOMEAS2",
                                "IDMN", "ID", "IDN", "IV", "JAVE", "JE", "JMAX", "SUMAVE", "SUMENT", "JVAR", "SUMVAR",
                                "VARIANCE")]
NGTDM = ["NGTDM_" + f for f in ("COARSENESS", "CONTRAST", "BUSYNESS", "COMPLEXITY", "STRENGTH")]
GLDM = ["GLDM_" + f for f in ("SDE", "LDE", "GLN", "DN", "DNN", "GLV", "DV", "DE", "LGLE", "HGLE", "SDLGLE", "SDHGLE",
                              "LDLGLE", "LDHGLE")]
GLRLM = ["GLRLM_" + f for f in ("SRE", "LRE", "GLNU", "GLNUN", "RLNU", "RLNUN", "RP", "GLV", "RV", "RE", "LGLRE",
                                "HGLRE", "SRLGLE", "SRHGLE", "LRLGLE", "LRHGLE")]
GLSZM = ["GLSZM_" + f for f in ("SAE", "LAE", "GLNU", "GLNUN", "SZNU", "SZNUN", "ZP", "GLV", "ZV", "ZE", "LGLZE",
                                "HGLZE", "SALGLE", "SAHGLE", "LALGLE", "LAHGLE", "GLM", "ZSM")]

# broad feature groups of the library (Table S1/S5 intensity, Table S2
# moments, Table S3 texture: GLCM, NGTDM, GLDM, GLRLM and GLSZM); together
# every feature
GROUPS = {
    "intensity": ["MEAN", "MIN", "MAX", "RANGE", "VARIANCE", "VARIANCE_BIASED", "STDDEV", "STDDEV_BIASED", "SKEWNESS",
                  "KURTOSIS", "EXCESS_KURTOSIS", "HYPERSKEWNESS", "HYPERFLATNESS", "ENERGY", "ROOT_MEAN_SQUARED",
                  "STANDARD_ERROR", "MEAN_ABSOLUTE_DEVIATION", "MEDIAN_ABSOLUTE_DEVIATION", "INTEGRATED_INTENSITY",
                  "WEIGHTED_CENTROID_X", "WEIGHTED_CENTROID_Y", "WEIGHTED_CENTROID_Z", "MASS_DISPLACEMENT", "COV",
                  "COVERED_IMAGE_INTENSITY_RANGE", "UNIFORMITY_PIU", "MEDIAN", "P01", "P10", "P25", "P75", "P90",
                  "P99", "INTERQUARTILE_RANGE", "QCOD", "ROBUST_MEAN", "ROBUST_MEAN_ABSOLUTE_DEVIATION", "MODE",
                  "MODE_PROBABILITY", "ENTROPY", "UNIFORMITY", "EDGE_INTEGRATED_INTENSITY", "EDGE_MAX_INTENSITY",
                  "EDGE_MIN_INTENSITY", "EDGE_MEAN_INTENSITY", "EDGE_STDDEV_INTENSITY"],
    "moments": ["INT_M", "INT_MU", "INT_ETA", "INT_NU", "INT_HU", "BIN_M", "BIN_MU", "BIN_ETA", "BIN_NU", "BIN_HU"],
    "texture": GLCM + NGTDM + GLDM + GLRLM + GLSZM,
}


def _extractor(w, features: Optional[Sequence[str]], max_rois: int):
    import torch

    from . import nyx

    dt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
    prm = w.params
    return nyx.Extractor(w.image.shape, dt, ndim=w.ndim, glcm_levels=prm["glcm_levels"], dists=prm["dists"],
                         hist_bins=prm["hist_bins"], features=features, max_rois=max_rois)


def time_device(w, features=None, steps: int = 10, warmup: int = 3) -> float:
    """Median ms of an extraction whose inputs are resident in HBM (CUDA
    events around each CUDA-graph replay)."""
    import torch

    mr = max(64, 2 * w.meta["n_roi"])
    ex = _extractor(w, features, mr)
    img = torch.from_numpy(w.image).cuda()
    mask = torch.from_numpy(w.mask).cuda()
    table = torch.empty((mr, len(ex.columns)), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        ex.extract_into(img, mask, table)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ex.extract_into(img, mask, table)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ex.sync_status()
    return float(np.median(ts))


def time_end_to_end(w, steps: int = 5, warmup: int = 2) -> Dict:
    """Median ms of pinned host image + mask -> device, extraction, and the
    table back to pinned host memory, on one stream; with the bytes moved."""
    import torch

    mr = max(64, 2 * w.meta["n_roi"])
    ex = _extractor(w, None, mr)
    h_img = torch.from_numpy(w.image).pin_memory()
    h_mask = torch.from_numpy(w.mask).pin_memory()
    d_img, d_mask = torch.empty_like(h_img, device="cuda"), torch.empty_like(h_mask, device="cuda")
    table = torch.empty((mr, len(ex.columns)), dtype=torch.float64, device="cuda")
    n = w.meta["n_roi"]
    h_table = torch.empty((n, len(ex.columns)), dtype=torch.float64).pin_memory()

    def step():
        d_img.copy_(h_img, non_blocking=True)
        d_mask.copy_(h_mask, non_blocking=True)
        ex.extract_into(d_img, d_mask, table)
        h_table.copy_(table[:n], non_blocking=True)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ex.sync_status()
    return {"ms": float(np.median(ts)), "h2d_bytes": int(w.image.nbytes + w.mask.nbytes),
            "d2h_bytes": int(h_table.numel() * 8)}


def family_costs(w, steps: int = 40) -> Dict[str, float]:
    """Device ms with the NGTDM, GLDM, GLRLM and GLSZM families removed from
    the full set and alone, which separates a family's own cost from its
    effect on the rest of the step."""
    base = GROUPS["intensity"] + GROUPS["moments"] + GLCM
    cases = {"all": None, "all_but_glrlm_glszm": base + NGTDM + GLDM, "all_but_gldm": base + NGTDM + GLRLM + GLSZM,
             "all_but_four": base, "gldm_only": GLDM, "ngtdm_only": NGTDM, "ngtdm_gldm": NGTDM + GLDM,
             "glrlm_only": GLRLM, "glszm_only": GLSZM, "glrlm_glszm": GLRLM + GLSZM,
             "intensity_only": GROUPS["intensity"]}
    return {k: time_device(w, v, steps=steps) for k, v in cases.items()}


def group_costs(w, steps: int = 10) -> Dict[str, float]:
    """Device ms of the extraction restricted to each feature group, and of
    all groups together."""
    out = {g: time_device(w, feats, steps=steps) for g, feats in GROUPS.items()}
    out["all"] = time_device(w, None, steps=steps)
    return out
