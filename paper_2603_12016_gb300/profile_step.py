"""One profiled extraction per synthetic workload, for ncu range capture.

    ncu --profile-from-start off --clock-control none --metrics ... \
        python -m paper_2603_12016_gb300.profile_step nuclei2d,ct3d,...

For each named workload: build an Extractor with the benchmark's settings
(the stored tuning of this device, else the default class limits), run three
warm-up extractions, then one more (forward + backward for the float batch)
between cudaProfilerStart and cudaProfilerStop, so that a profiler started
with capture off records exactly that extraction's launches.  The hot-path
feature set is used for the 2048² nuclei workload (as in the benchmark's
headline line; --all selects the full set there too), the full set
elsewhere.

    python -m paper_2603_12016_gb300.profile_step nuclei2d --subsets

instead profiles one extraction of the named workload per feature
subset (MEAN alone, then MEAN plus one feature family), with the class
limits of the hot-path set; the differences of the per-kernel instruction
counts attribute the fused kernel's work to the families.

    --scan-staging=0|1 overrides the stored label-scan row staging (0 bulk
    tensor copies where the row pitch allows, 1 register loads).
"""
from __future__ import annotations

import os
import sys


SUBSETS = (("base", ["MEAN"]), ("order", ["MEAN", "MEDIAN"]), ("histogram", ["MEAN", "ENTROPY"]),
           ("moments", ["MEAN", "INT_M", "BIN_M"]), ("glcm", ["MEAN", "GLCM_ASM"]),
           ("ngtdm", ["MEAN", "NGTDM_COARSENESS"]), ("gldm", ["MEAN", "GLDM_SDE"]), ("glrlm", ["MEAN", "GLRLM_SRE"]),
           ("glszm", ["MEAN", "GLSZM_SAE"]), ("core", "core"),
           ("all", None))


def _profiled(ex, img, mask, table, bwd=False, g=None):
    import torch

    for i in range(4):
        if i == 3:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        ex.extract_into(img, mask, table, save_for_backward=bwd)
        if bwd:
            ex.backward(img, mask, g)
        if i == 3:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    ex.sync_status()


def main(argv=None) -> int:
    import numpy as np
    import torch

    from . import build, nyx, tuning
    from . import workloads as W

    argv = sys.argv[1:] if argv is None else argv
    subsets = "--subsets" in argv
    full = "--all" in argv  # the full feature set for the 2048^2 nuclei workload too
    stg = [int(a.split("=", 1)[1]) for a in argv if a.startswith("--scan-staging=")]
    stg = stg[-1] if stg else None
    argv = [a for a in argv if a not in ("--subsets", "--all") and not a.startswith("--scan-staging=")]
    names = (argv[0] if argv else "nuclei2d").split(",")
    procs = max(1, min(16, os.cpu_count() or 1))
    # build every workload before the first CUDA call (the mosaic's tiles use spawned processes)
    wl = {n: (W.mosaic_workload(n, 0, procs) if n.startswith("mosaic") else W.config(n)) for n in names}
    build.build()
    torch.cuda.set_device(0)
    dev = torch.cuda.get_device_name(0)
    if subsets:
        w = wl[names[0]]
        prm = w.params
        img, mask = torch.from_numpy(w.image).cuda(), torch.from_numpy(w.mask).cuda()
        sig = tuning.signature(w.image.shape, str(w.image.dtype), w.ndim, prm["glcm_levels"], prm["dists"], "core")
        for name, f in SUBSETS:
            tdt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
            ex = nyx.Extractor(w.image.shape, tdt, ndim=w.ndim, glcm_levels=prm["glcm_levels"],
                               dists=prm["dists"], hist_bins=prm["hist_bins"], max_rois=8192,
                               features=nyx.CORE_FEATURE_IDS if f == "core" else f)
            t, _ = tuning.limits_for(ex, dev, sig)
            table = torch.empty((ex.max_rois, len(ex.columns)), dtype=torch.float64, device="cuda")
            _profiled(ex, img, mask, table)
            print(name, len(ex.columns), t, flush=True)
            del ex, table
        return 0
    for n, w in wl.items():
        feats = "core" if n == "nuclei2d" and not full else "all"
        prm = w.params
        tdt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
        nr = w.meta["n_roi"]
        ex = nyx.Extractor(w.image.shape, tdt, ndim=w.ndim, glcm_levels=prm["glcm_levels"], dists=prm["dists"],
                           hist_bins=prm["hist_bins"], max_rois=8192 if nr <= 8192 else 2 * nr,
                           features=nyx.CORE_FEATURE_IDS if feats == "core" else None)
        sig = tuning.signature(w.image.shape, str(w.image.dtype), w.ndim, prm["glcm_levels"], prm["dists"], feats)
        t, src = tuning.limits_for(ex, dev, sig)
        if stg is not None:
            ex.set_scan_staging(stg)
            t = ex.tuning()
        img, mask = torch.from_numpy(w.image).cuda(), torch.from_numpy(w.mask).cuda()
        bwd = n.startswith("blobbatch")
        table = torch.empty((ex.max_rois, len(ex.columns)), dtype=torch.float64, device="cuda")
        g = torch.zeros_like(table) if bwd else None
        _profiled(ex, img, mask, table, bwd, g)
        print(n, feats, t, src, flush=True)
        del ex, img, mask, table
        torch.cuda.empty_cache()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
