"""Autotuned size-class limits, persisted per device and workload.

The per-ROI kernels come in four size classes (one warp per ROI, a small
block, a medium block, several blocks per ROI).  Which ROI goes to which
class is decided by pixel limits; the best limits depend on the GPU and on
the workload's ROI size distribution ("Results, Scalability": ROI size decides
where a GPU pays off).  The label scan's tile shape (128 columns by 64, 128
or 256 rows) and how it stages its rows (bulk tensor copies or register
loads) are the other tuned launch parameters.  `tune` runs the library's
autotuner (nyx_autotune: every candidate timed with the L2 cache flushed
before each call) on a given input.  Results are stored in tuned.json next to
this file, keyed by the device name and a workload signature (image shape,
pixel type, grey levels, distances, feature selection), so that the
benchmark and `Extractor` users get the same, reproducible launch
configuration without tuning at run time.

    python -m paper_2603_12016_gb300.tuning [--workloads nuclei2d,ct3d,...]

runs the tuner on the named synthetic workloads and rewrites the entries of
the current device (the file's other entries are kept).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
from typing import Dict, Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
TUNED_PATH = os.path.join(HERE, "tuned.json")
DEFAULT_LIMITS = (256, 1024, 4096, 8192)  # warp, small, medium, large block classes


def signature(shape: Sequence[int], dtype: str, ndim: int, ng: int, dists: Sequence[int], features: str) -> str:
    return (f"{'x'.join(str(int(s)) for s in shape)}|{dtype}|{ndim}d|ng{int(ng)}|"
            f"d{','.join(str(int(d)) for d in dists)}|{features}")


def _read(path: str = TUNED_PATH) -> Dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def load(device_name: str, sig: str, path: str = TUNED_PATH) -> Optional[Dict]:
    """The stored entry ({"limits": [w, s, m, l], "scan_rows_per_warp": r, "scan_staging": g, "ms": ...})
    or None."""
    return _read(path).get(device_name, {}).get(sig)


def store(device_name: str, sig: str, entry: Dict, path: str = TUNED_PATH) -> None:
    d = _read(path)
    d.setdefault(device_name, {})[sig] = entry
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)


def time_config(ex, img, mask, table, steps: int = 10, warmup: int = 3) -> float:
    """Median device time (ms) of graph-replayed extractions with the plan's
    current settings, L2 flushed before every timed step."""
    import torch

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=img.device)
    stream = torch.cuda.current_stream(img.device)
    for _ in range(warmup):
        ex.extract_into(img, mask, table)
    ex.sync_status()
    ts = []
    for _ in range(steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        ex.extract_into(img, mask, table)
        e.record(stream)
        e.synchronize()
        ts.append(s.elapsed_time(e))
    ex.sync_status()
    return statistics.median(ts)


def tune(ex, img, mask, reps: int = 5) -> Tuple[Tuple[int, ...], float]:
    """The library's autotuner (nyx_autotune: class limits, then the label
    scan's tile height, each candidate the median of `reps` L2-flushed
    calls) on this input; returns the setting and its median time."""
    import torch

    t = ex.autotune(img, mask, reps=reps)
    table = torch.empty((ex.max_rois, len(ex.columns)), dtype=torch.float64, device=img.device)
    return t, time_config(ex, img, mask, table)


def limits_for(ex, device_name: str, sig: str) -> Tuple[Tuple[int, ...], str]:
    """Apply the stored setting of (device, workload) to `ex` if there is
    one; returns the setting in force and where it came from."""
    ent = load(device_name, sig)
    if ent:
        t = tuple(int(v) for v in ent["limits"]) + (int(ent.get("scan_rows_per_warp", 0)),
                                                      int(ent.get("scan_staging", 0)))
        ex.set_tuning(*t)
        return t, "tuned.json"
    t = DEFAULT_LIMITS + (0, 0)
    ex.set_tuning(*t)
    return t, "default"


def main() -> int:
    import numpy as np
    import torch

    from . import build, nyx
    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="nuclei2d,ct3d,blobbatch,mosaic_small")
    ap.add_argument("--features", default="core,all")
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    procs = max(1, min(16, os.cpu_count() or 1))
    wl = {name: (W.mosaic_workload(name, 0, procs) if name.startswith("mosaic") else W.config(name))
          for name in a.workloads.split(",")}  # before any CUDA call (the mosaic's tiles use spawned processes)
    build.build()
    torch.cuda.set_device(0)
    dev_name = torch.cuda.get_device_name(0)
    for name, w in wl.items():
        img_np, mask_np, ndim, prm = w.image, w.mask, w.ndim, w.params
        tdt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[img_np.dtype.type]
        n_roi = int(np.count_nonzero(np.bincount(mask_np.ravel())[1:]))
        for feats in a.features.split(","):
            ex = nyx.Extractor(img_np.shape, tdt, ndim=ndim, glcm_levels=prm["glcm_levels"], dists=prm["dists"],
                               hist_bins=prm["hist_bins"], max_rois=8192 if n_roi <= 8192 else 2 * n_roi,
                               features=nyx.CORE_FEATURE_IDS if feats == "core" else None)
            img = torch.from_numpy(img_np).cuda()
            mask = torch.from_numpy(mask_np).cuda()
            t, ms = tune(ex, img, mask, reps=a.reps)
            sig = signature(img_np.shape, str(img_np.dtype), ndim, prm["glcm_levels"], prm["dists"], feats)
            store(dev_name, sig, {"limits": list(t[:4]), "scan_rows_per_warp": t[4], "scan_staging": t[5],
                                  "ms": round(ms, 4),
                                  "how": "nyx_autotune (median of L2-flushed calls per candidate), then the "
                                         "median of 10 L2-flushed graph replays of the choice"})
            print(json.dumps({"workload": name, "features": feats, "tuning": t, "ms": round(ms, 4)}), flush=True)
            del ex
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
