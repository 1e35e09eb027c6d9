#!/usr/bin/env python
"""Benchmark of batched per-ROI feature extraction on GB300.

Workload (default): one 2048x2048 uint16 fluorescence-like image with ~3600
ROIs of 50-4100 px (seeded synthetic stand-in for TissueNet), full feature
set: first-order statistics, order statistics, histogram features, raw /
central / normalised moments with Hu invariants (intensity and binary), GLCM
with 256 grey levels at distances 1 and 2 over 4 directions.

A step is one nyx_extract over the device-resident image (label scan, key
sort, per-ROI feature kernels, table reset).  L2 (129 MB) is flushed by
writing a 256 MB buffer between timed steps because the input (25 MB) fits
in L2.  Times are CUDA events on the launching stream; with N ranks every
rank processes its own image (independent problems, weak scaling) and rank 0
reports the maximum time over ranks.

--impl reference times the CPU FP64 oracle (the only reference this paper
offers) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ROIs/sec and Mpixel/sec full feature set, % HBM roofline vs plain FP64 path"
PHASES = ("scan", "sort_setup", "roi_warp", "roi_small", "roi_medium", "roi_big", "final", "reset")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) taken every
    20 ms while the timed regions run; each sample is tagged with the region
    (workload) that was being timed when it arrived."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.tag = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8 and self.tag is not None:
                self.rows.append([self.tag] + parts)

    def region(self, tag):
        sampler = self

        class _R:
            def __enter__(self):
                sampler.tag = tag
                time.sleep(0.05)  # let the sampler see the start of the region

            def __exit__(self, *a):
                sampler.tag = None

        return _R()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stats(rows):
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        out = self._stats(self.rows)
        out["by_region"] = {t: self._stats([r for r in self.rows if r[0] == t])
                            for t in dict.fromkeys(r[0] for r in self.rows)}
        return out


# DRAM bytes (read + write) per launch of a phase's kernel, from one ncu
# capture of the same bench command, keyed by workload, phase, class limits
# with the scan's tile height and row staging, and feature set, and valid only for the kernel sources they were taken
# with (the hash below; any change to csrc/ voids them and traffic is null).
# ROI-stage traffic (DRAM read + write of every k_roi class, multi-block
# kernel and GLRLM / GLSZM kernel of one extraction, ncu --profile-from-start
# off over python -m paper_2603_12016_gb300.profile_step <workload>), plus
# the one clear of the GLRLM / GLSZM per-pixel arrays (12 bytes a pixel,
# a memset ncu does not list).  The 32768^2 mosaic is scaled from the 8192^2
# mosaic: kernel bytes by ROI pixels (565.05M / 36.02M), the clear by
# image pixels.
TRAFFIC_SRC = "c39cc1dc7bf2efff"
TRAFFIC = {
    ("nuclei2d_2048_u16_4000roi", "roi_stage", (256, 1024, 4096, 8192, 8, 1), "core"): 36.26e6,
    ("ct3d_512x512x128_i16_200roi", "roi_stage", (0, 1024, 2048, 8192, 32, 0), "all"): 3527.77e6 + 12 * 512 * 512 * 128,
    ("blobbatch_64x512_f32", "roi_stage", (0, 1024, 4096, 8192, 16, 0), "all"): 108.23e6,
    ("mosaic_32768_u16_500000roi", "roi_stage", (0, 512, 4096, 8192, 32, 0), "all"): 1335.98e6 * 565.05 / 36.02
    + 12 * 32768 * 32768,
}


def kernel_source_hash() -> str:
    """Hash of the CUDA sources the library is built from, comments and
    whitespace removed (an edit of a comment leaves the kernels unchanged)."""
    import glob
    import hashlib
    import re

    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2603_12016_gb300", "csrc", "*.cu*"))):
        with open(f, encoding="utf-8") as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(os.path.basename(f).encode() + " ".join(code.split()).encode())
    return h.hexdigest()[:16]


def roi_classes(w, lim_pix):
    """Pixels and ROI count per size class (warp, small, medium, large,
    multi-block) by the library's class rule: pixel count against the class
    limits and padded bounding-box cells against the class capacities 1,024
    / 4,096 / 8,192 / 16,384."""
    from scipy import ndimage

    pad = max(w.params["dists"])  # the plan pads every raster by the largest distance (>= 1)
    lims = tuple(zip(lim_pix, (1024, 4096, 8192, 16384)))
    nc = len(lims)
    px, rows = [0] * (nc + 1), [0] * (nc + 1)
    masks = w.mask.reshape((-1,) + w.mask.shape[-w.ndim:]) if w.mask.ndim > w.ndim else w.mask[None]
    for m in masks:
        cnt = np.bincount(m.ravel())
        for lab, sl in enumerate(ndimage.find_objects(m), start=1):
            if sl is None:
                continue
            ext = [s.stop - s.start + 2 * pad for s in sl]
            cells = int(np.prod(ext))
            n = int(cnt[lab])
            k = nc
            for i in range(nc - 1, -1, -1):
                if n <= lims[i][0] and cells <= lims[i][1]:
                    k = i
            px[k] += n
            rows[k] += 1
    return px, rows


def reduce_over_ranks(dist, device, t_ms: float, units: int):
    """Whole-job figures of independent per-rank problems (weak scaling, no
    collective on the data path): the slowest rank's time and the units that
    all ranks processed."""
    if dist is None:
        return t_ms, units
    import torch

    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    nn = torch.tensor([units], dtype=torch.int64, device=device)
    dist.all_reduce(nn)
    return float(tt.item()), int(nn.item())


def make_workload(name: str, rank: int, procs: int = 1):
    from paper_2603_12016_gb300 import workloads as W

    if name.startswith("mosaic"):
        # whole-slide stand-in generated tile by tile (tiles in parallel
        # processes, started with spawn before any CUDA call); the assembled
        # arrays are what the host streams
        return W.mosaic_workload(name, rank, procs)
    return W.config(name, seed_offset=rank)


def algorithmic_bytes(w, n_roi: int, n_col: int) -> int:
    """Each input byte read once plus the FP64 table written once."""
    return int(w.image.nbytes + w.mask.nbytes + 8 * n_roi * n_col)


def run_reference(args) -> int:
    """CPU FP64 oracle on a bounded sample of the workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle

    w = make_workload(args.workload, 0)
    cores = os.cpu_count() or 1
    image, mask, where = _oracle_view(w)
    labels = _roi_keys(w, mask)
    sample = labels[: min(len(labels), args.ref_rois)]
    keys = [int(k) for k in sample]
    prm = w.params
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.extract(image, mask, w.ndim, ng=prm["glcm_levels"], dists=prm["dists"],
                       hist_bins=prm["hist_bins"], rois=keys, threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    v = len(sample) / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ROIs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample_rois": int(len(sample)), "n_roi_total": int(len(labels)),
                       "glcm_levels": prm["glcm_levels"], "dists": list(prm["dists"])},
            "cpu_baseline": {"value": v, "unit": "ROIs/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {len(sample)} of {len(labels)} ROIs of {w.name}{where}"},
            "e2e": {"value": v, "unit": "ROIs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _roi_keys(w, mask):
    """Oracle ROI keys (image << 32 | label) of every ROI, ascending."""
    import oracle

    per = mask.reshape((-1,) + mask.shape[-w.ndim:]) if mask.ndim > w.ndim else mask[None]
    return [oracle.roi_key(b, int(l)) for b, m in enumerate(per) for l in np.unique(m[m > 0])]


def _oracle_view(w):
    """Arrays the oracle samples from: the first 4096 x 4096 tile of a
    streamed mosaic (the oracle separates every pixel of its input first),
    else the whole workload."""
    if w.meta.get("tile"):
        return w.image[:4096, :4096], w.mask[:4096, :4096], " (first 4096x4096 tile)"
    return w.image, w.mask, ""


def cpu_baseline(w, budget_s: float, note: str = ""):
    """Time the oracle on the host cores on a bounded ROI sample."""
    import numpy as np
    import oracle

    cores = os.cpu_count() or 1
    image, mask, where = _oracle_view(w)
    labels = _roi_keys(w, mask)
    prm = w.params
    n = 32
    while True:
        sample = labels[: min(n, len(labels))]
        keys = [int(k) for k in sample]
        t0 = time.perf_counter()
        oracle.extract(image, mask, w.ndim, ng=prm["glcm_levels"], dists=prm["dists"],
                       hist_bins=prm["hist_bins"], rois=keys, threads=cores)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or len(sample) == len(labels):
            break
        n = int(n * min(8.0, max(2.0, budget_s / 4 / max(dt, 1e-3))))
    return {"value": len(sample) / dt, "unit": "ROIs/s", "cores": cores, "kind": "oracle",
            "sample": f"first {len(sample)} of {len(labels)} ROIs of {w.name}{where}, {dt:.1f} s"
                      + (f"; oracle computes {note}" if note else ""),
            "seconds": dt}


def _oracle_ms(w, budget_s: float):
    """CPU oracle time for all of w's ROIs, extrapolated from a bounded
    sample of them (all host cores); the sample size is returned too."""
    import numpy as np
    import oracle

    cores = os.cpu_count() or 1
    labels = np.unique(w.mask[w.mask > 0])
    prm = w.params
    n = min(8, len(labels))
    while True:
        keys = [oracle.roi_key(0, int(l)) for l in labels[:n]]
        t0 = time.perf_counter()
        oracle.extract(w.image, w.mask, w.ndim, ng=prm["glcm_levels"], dists=prm["dists"],
                       hist_bins=prm["hist_bins"], rois=keys, threads=cores)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or n == len(labels):
            break
        n = min(len(labels), int(n * min(8.0, max(2.0, budget_s / 4 / max(dt, 1e-3)))))
    return 1e3 * dt * len(labels) / n, n, cores


def run_scalability_sweep(args) -> int:
    """Time over ROI size x ROI count (the study of Fig. 3f): GPU with inputs
    in HBM, GPU end to end from pinned host buffers, and the CPU oracle on a
    bounded sample scaled to all ROIs; then the per-group cost structure of
    an image of 100 ROIs of 100,000 px (Fig. 3g)."""
    import torch

    from paper_2603_12016_gb300 import scalability as S
    from paper_2603_12016_gb300 import workloads as W

    torch.cuda.set_device(0)
    rows = []
    for n_roi in (10, 100, 1000):
        for px in (100, 500, 1000, 5000, 20000, 100000):
            w = W.scalability_2d(px, n_roi)
            dev = S.time_device(w, steps=10)
            e2e = S.time_end_to_end(w)
            ora, ns, cores = _oracle_ms(w, budget_s=2.0)
            rows.append({"roi_px": px, "n_roi": w.meta["n_roi"], "image": list(w.image.shape),
                         "gpu_ms": round(dev, 4), "gpu_e2e_ms": round(e2e["ms"], 4), "h2d_bytes": e2e["h2d_bytes"],
                         "oracle_ms": round(ora, 2), "oracle_sample_rois": ns, "oracle_cores": cores})
    w = W.scalability_2d(100000, 100)
    groups = S.group_costs(w)
    ora, ns, cores = _oracle_ms(w, budget_s=6.0)
    print(json.dumps({"metric": "scalability over ROI size x count; feature-group cost of 100 x 100,000 px",
                      "unit": "ms", "features": "all", "rows": rows,
                      "cost_100x100k": {"gpu_ms": {k: round(v, 4) for k, v in groups.items()},
                                        "oracle_ms": round(ora, 1), "oracle_sample_rois": ns,
                                        "oracle_cores": cores}}))
    return 0


def run_family_sweep(args) -> int:
    """Device ms of one extraction of the workload with the NGTDM, GLDM,
    GLRLM and GLSZM families removed from the full feature set and alone."""
    import torch

    from paper_2603_12016_gb300 import scalability as S
    from paper_2603_12016_gb300 import workloads as W

    torch.cuda.set_device(0)
    w = W.config(args.workload)
    out = S.family_costs(w, steps=max(args.steps // 5, 20))
    print(json.dumps({"metric": "feature-family cost (device ms per extraction, no L2 flush)", "unit": "ms",
                      "workload": w.name, "ms": {k: round(v, 4) for k, v in out.items()}}))
    return 0


def run_soft_sweep(args) -> int:
    """GLCM soft-feature grid: compute time over grey depth (Eq. 2) x nested
    distance sets (Eq. 3), checked for the ordering of Eq. 5, and the Eq. 8
    separability ratio of every GLCM feature over the same grid on labelled
    synthetic texture classes."""
    import torch

    from paper_2603_12016_gb300 import softgrid
    from paper_2603_12016_gb300 import workloads as W

    torch.cuda.set_device(0)
    levels = [16, 32, 64, 128, 256]
    dist_sets = [[1], [1, 2], [1, 2, 3], [1, 2, 3, 4]]
    w = W.config("nuclei2d")
    t = softgrid.timing_grid(w, levels, dist_sets, steps=max(args.steps // 10, 10), warmup=args.warmup)
    mono = softgrid.monotone_report(t)
    tw = W.texture_classes_2d()
    sep = softgrid.separability_grid(tw, tw.meta["classes"], levels, dist_sets)
    top = sorted(sep["best_point"].items(), key=lambda kv: -kv[1]["ratio"])[:5]
    print(json.dumps({
        "metric": "GLCM soft-feature grid (Eqs. 2-5) and Eq. 8 separability", "unit": "ms",
        "workload": w.name, "features": "GLCM only", "levels": levels, "dist_sets": dist_sets,
        "ms": [[round(x, 4) for x in row] for row in t.tolist()],
        "monotone": {"steps": mono["steps"], "holds": mono["holds"], "violations": mono["violations"]},
        "separability_workload": tw.name, "top_features": [{"feature": f, **v} for f, v in top],
        "best_feature_by_point": sep["best_feature"]}))
    return 0


EXTRA_CONFIGS = ("ct3d", "blobbatch", "mosaic")  # measured beside the headline, in sub-objects


def run_config(name, w, dev, dist, args, features, clk, light=False, flush=None):
    """Time one workload: CUDA-graph replay of nyx_extract (+ nyx_backward for
    the differentiation workload) over device-resident inputs, L2 flushed
    before every step; per-phase device times from the event nodes inside
    the replayed graph; the dominant kernel's roofline; end to end through
    the public API from pinned host memory.  Returns the measurement dict."""
    import torch

    from paper_2603_12016_gb300 import nyx, tuning

    prm = w.params
    dtype = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
    max_rois = 8192 if w.meta["n_roi"] <= 8192 else 2 * w.meta["n_roi"]
    tile = w.meta.get("tile")
    feats = nyx.CORE_FEATURE_IDS if features == "core" else None

    def extractor(precision):
        return nyx.Extractor(w.image.shape, dtype, ndim=w.ndim, glcm_levels=prm["glcm_levels"], dists=prm["dists"],
                             hist_bins=prm["hist_bins"], precision=precision, max_rois=max_rois, device=dev,
                             features=feats)

    ex = extractor("fp32")
    sig = tuning.signature(w.image.shape, str(w.image.dtype), w.ndim, prm["glcm_levels"], prm["dists"], features)
    dev_name = torch.cuda.get_device_name(dev)
    if args.class_limits:
        limits = tuple(int(v) for v in args.class_limits.split(","))
        limits, lim_src = (limits + (0, 0))[:6], "command line"
        ex.set_tuning(*limits)
    else:
        limits, lim_src = tuning.limits_for(ex, dev_name, sig)
    img = torch.from_numpy(w.image).to(dev)
    mask = torch.from_numpy(w.mask).to(dev)
    n_col = len(ex.columns)
    table = torch.empty((max_rois, n_col), dtype=torch.float64, device=dev)
    if flush is None:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    bwd = name.startswith("blobbatch") if args.backward is None else args.backward
    gen = torch.Generator(device=dev).manual_seed(5)
    gtab = torch.randn((max_rois, n_col), dtype=torch.float64, device=dev, generator=gen) if bwd else None
    gimg = torch.empty(img.shape, dtype=torch.float32, device=dev) if bwd else None

    def one_step(e, im, mk, bwd_ev=None):
        n = e.extract_into(im, mk, table, save_for_backward=bwd)
        if bwd:
            if bwd_ev:
                bwd_ev[0].record(stream)
            e.backward(im, mk, gtab, out=gimg)
            if bwd_ev:
                bwd_ev[1].record(stream)
        return n

    def timed(e, steps, warmup, phases=True):
        """Per-step device times (CUDA events on the launching stream) and,
        with phases, the per-phase times of each step's graph replay."""
        e.graph_phase_events(phases)
        for _ in range(warmup):
            one_step(e, img, mask)
        e.sync_status()
        ms, ph = [], []
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        n = None
        for i in range(steps):
            flush.zero_()
            s_, t_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            bev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) if bwd else None
            s_.record(stream)
            n = one_step(e, img, mask, bev)
            t_.record(stream)
            t_.synchronize()
            ms.append(s_.elapsed_time(t_))
            if phases:
                d = e.graph_phase_times()
                if bwd:
                    d["backward"] = bev[0].elapsed_time(bev[1])
                ph.append(d)
        torch.cuda.synchronize(dev)
        e.sync_status()
        e.graph_phase_events(False)
        return ms, ph, int(n.item())

    with clk.region(name + ("" if features == "all" else "/" + features)):
        ms, ph, n_roi = timed(ex, args.steps, args.warmup)
    t_step, n_total = reduce_over_ranks(dist, dev, statistics.median(ms), n_roi)
    phases = {k: sum(p[k] for p in ph) / len(ph) for k in ph[0]}
    res = {"workload": w.name, "features": features, "n_roi": n_roi, "n_col": n_col,
           "value": n_total / (t_step * 1e-3), "unit": "ROIs/s", "ms_per_step": t_step,
           "step": "forward + backward" if bwd else "forward",
           "class_limits_px": list(limits[:4]), "scan_rows_per_warp": limits[4], "scan_staging": limits[5],
           "class_limits_source": lim_src,
           "mpix_per_s": w.image.size * (dist.get_world_size() if dist else 1) / (t_step * 1e-3) / 1e6,
           "phases_ms": {k: round(v, 5) for k, v in phases.items()}}
    if light:
        return res

    # dominant kernel (longest phase of the replayed graph) and its roofline:
    # algorithmic bytes per launch (the scan streams image + mask once; a ROI
    # class reads its ROIs' pixels and mask once and writes their table rows;
    # the backward pass reads image + mask and writes the gradient)
    cls_px, cls_rows = roi_classes(w, limits[:4])
    n_off = len(prm["dists"]) * (13 if w.ndim == 3 else 4) if prm["glcm_levels"] > 0 else 0
    per_px = w.image.itemsize + 4
    # The four size classes run as concurrent graph branches, each holding SMs
    # the others wait for, so a class's own span is not its kernel time; the
    # per-ROI stage (fork to join) is timed as one unit with the bytes of
    # every ROI pixel and table row.
    alg_by_phase = {"scan": w.image.nbytes + w.mask.nbytes,
                    "roi_stage": sum(cls_px) * per_px + 8 * n_roi * n_col,
                    "glcm_final": n_roi * n_off * 160,
                    "stats_final": n_roi * 512,
                    "backward": w.image.nbytes + w.mask.nbytes + 4 * w.image.size}
    cand = {k: v for k, v in phases.items() if k in alg_by_phase}
    dom = max(cand, key=cand.get)
    dom_bytes = alg_by_phase[dom]
    dom_gbs = dom_bytes / (phases[dom] * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    src = kernel_source_hash()
    tr = TRAFFIC.get((w.name, dom, tuple(limits), features)) if TRAFFIC_SRC == src else None
    kern = {"roi_stage": "per-ROI stage: k_roi warp/small/medium classes + multi-block kernels, concurrent",
            "scan": "k_scan_tma (label scan, bulk-copy staged; k_scan where the row pitch rules it out)",
            "backward": "k_bwd_coef + k_bwd_pixel",
            "glcm_final": "k_glcm_final", "stats_final": "k_stats_final"}[dom]
    res["roofline"] = {"bound": "hbm", "kernel": kern, "phase": dom, "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                       "frac": dom_gbs / peak, "traffic": tr, "peak_kind": peak_kind,
                       "algorithmic_bytes": int(dom_bytes), "avg_launch_ms": phases[dom],
                       "timing": "CUDA event nodes inside each timed graph replay, on the kernel's own stream"}
    alg = algorithmic_bytes(w, n_roi, n_col) + (4 * w.image.size if bwd else 0)
    res["pipeline_hbm"] = {"algorithmic_bytes": alg, "achieved_gbs": alg / (t_step * 1e-3) / 1e9,
                           "frac": alg / (t_step * 1e-3) / 1e9 / peak, "peak": peak, "peak_kind": peak_kind}
    res["roi_mpix_per_s"] = float((w.mask > 0).sum()) / (t_step * 1e-3) / 1e6
    res["l2"] = "flushed (256 MB write) before every step"
    # our kernels per step: front (counters + scan), key sort, setup; the
    # block classes with a nonzero limit; the multi-block path (zero, pass 1,
    # pass 2, order statistics, + GLCM, + neighbour kernel); GLCM features;
    # statistics; reset; backward: coefficients + per-pixel gradient + reset
    glcm = prm["glcm_levels"] > 0
    n_cls = sum(1 for v in limits[:4] if v > 0)
    per_step = 3 + n_cls + 4 + (2 if glcm else 0) + (1 if glcm else 0) + 1 + 1 + (3 if bwd else 0)
    res["gpu_launches"] = per_step * args.steps

    # end to end through the public API: pinned host inputs -> H2D -> extract -> D2H
    h_img = torch.from_numpy(w.image).pin_memory()
    h_mask = torch.from_numpy(w.mask).pin_memory()
    h_table = torch.empty((max_rois, n_col), dtype=torch.float64).pin_memory()
    h_grad = torch.empty(img.shape, dtype=torch.float32).pin_memory() if bwd else None
    d_img = torch.empty_like(img)
    d_mask = torch.empty_like(mask)
    e2e_ms = []
    h_img_np, h_mask_np = h_img.numpy(), h_mask.numpy()

    def tile_source(x0, y0, tw, th):
        return h_img_np[y0:y0 + th, x0:x0 + tw], h_mask_np[y0:y0 + th, x0:x0 + tw]

    e2e_steps = args.steps if tile is None else min(args.steps, 3)
    for i in range(args.warmup + e2e_steps):
        torch.cuda.synchronize(dev)
        s_, t_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record(stream)
        if tile is None:
            d_img.copy_(h_img, non_blocking=True)
            d_mask.copy_(h_mask, non_blocking=True)
            one_step(ex, d_img, d_mask)
        else:  # tiles streamed from host memory, band scans overlapping the host
            ex.extract_tiles(tile_source, (tile, tile), d_img, d_mask, table=table)
        h_table[:n_roi].copy_(table[:n_roi], non_blocking=True)
        if bwd:
            h_grad.copy_(gimg, non_blocking=True)
        t_.record(stream)
        t_.synchronize()
        if i >= args.warmup:
            e2e_ms.append(s_.elapsed_time(t_))
    e2e_t, _ = reduce_over_ranks(dist, dev, statistics.median(e2e_ms), n_roi)
    res["e2e"] = {"value": n_total / (e2e_t * 1e-3), "unit": "ROIs/s",
                  "h2d_bytes_per_step": int(w.image.nbytes + w.mask.nbytes),
                  "api": "nyx_extract_tiles" if tile else "nyx_extract",
                  "d2h_bytes_per_step": int(8 * n_roi * n_col + (4 * w.image.size if bwd else 0)),
                  "ms_per_step": e2e_t}
    del h_img, h_mask, h_table, h_grad, d_img, d_mask
    if not args.no_fp64:
        ex64 = extractor("fp64")
        ex64.set_tuning(*limits)
        ms64, _, _ = timed(ex64, max(3, args.steps // 4), 3, phases=False)
        t64 = statistics.median(ms64)
        res["fp64_plain"] = {"value": n_roi / (t64 * 1e-3), "unit": "ROIs/s", "ms_per_step": t64,
                             "speedup_fp32_over_fp64": t64 / t_step}
        del ex64
    return res


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nuclei2d")
    ap.add_argument("--configs", default=",".join(EXTRA_CONFIGS),
                    help="workloads measured beside the headline (comma list, '' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison path")
    ap.add_argument("--ref-rois", type=int, default=800)
    ap.add_argument("--backward", dest="backward", action="store_true", default=None,
                    help="time forward + backward (default for the blobbatch workloads)")
    ap.add_argument("--no-backward", dest="backward", action="store_false")
    ap.add_argument("--class-limits", default=None,
                    help="warp,small,medium,large pixel limits[,scan rows per warp[,scan staging 0 TMA / 1 "
                         "register loads]] instead of the tuned ones")
    ap.add_argument("--sweep", default=None, choices=["soft", "scalability", "families"],
                    help="soft: the GLCM timing grid of Eqs. 2-5 on the 2048^2 nuclei workload and the Eq. 8 "
                         "separability grid on labelled texture classes; scalability: time over ROI size x ROI "
                         "count (GPU device, GPU end to end, CPU oracle) and the feature-group cost of an image "
                         "of 100 ROIs of 100,000 px; families: the workload with the NGTDM, GLDM, GLRLM and "
                         "GLSZM families removed and alone (one JSON line each, not bench lines)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep == "soft":
        return run_soft_sweep(args)
    if args.sweep == "scalability":
        return run_scalability_sweep(args)
    if args.sweep == "families":
        return run_family_sweep(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    extra = [c for c in args.configs.split(",") if c]
    # workloads first: the mosaic's tiles are generated in spawned processes,
    # before this process makes any CUDA call
    procs = max(1, min(16, (os.cpu_count() or 1) // max(1, world)))
    wl = {name: make_workload(name, rank, procs) for name in [args.workload] + extra}

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2603_12016_gb300 import build

    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clk = ClockSampler(local)
    with clk:
        head = run_config(args.workload, wl[args.workload], dev, dist, args, "core", clk, flush=flush)
        allf = run_config(args.workload, wl[args.workload], dev, dist, args, "all", clk, light=True, flush=flush)
        subs = {}
        for name in extra:
            subs[name] = run_config(name, wl[name], dev, dist, args, "all", clk, flush=flush)
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    if not args.no_cpu_baseline and world == 1:
        head["cpu_baseline"] = cpu_baseline(wl[args.workload], 20.0, "all families (a superset of the timed set)")
        for name in extra:
            subs[name]["cpu_baseline"] = cpu_baseline(wl[name], 8.0, "all families")
    w = wl[args.workload]
    prm = w.params
    line = {
        "metric": METRIC, "value": head["value"], "unit": "ROIs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
        "config": {"workload": w.name, "image": list(w.image.shape), "pixel_dtype": str(w.image.dtype),
                   "n_roi": head["n_roi"], "n_col": head["n_col"], "glcm_levels": prm["glcm_levels"],
                   "dists": list(prm["dists"]), "hist_bins": prm["hist_bins"],
                   "features": "hot-path set: first-order + order statistics, histogram, raw/central/normalised "
                               "moments + Hu (intensity and binary), GLCM (30 features, direction means)",
                   "step": head["step"], "l2": head["l2"], "class_limits_px": head["class_limits_px"],
                   "scan_rows_per_warp": head["scan_rows_per_warp"],
                   "scan_staging": ["bulk tensor copies (TMA) where the row pitch allows",
                                    "register loads"][head["scan_staging"]],
                   "class_limits_source": head["class_limits_source"],
                   "timing": "median of per-step CUDA-event times, CUDA-graph replay",
                   "parallelism": f"replicas{world}"},
        "mpix_per_s": head["mpix_per_s"], "roi_mpix_per_s": head["roi_mpix_per_s"],
        "pipeline_hbm": head["pipeline_hbm"], "phases_ms": head["phases_ms"], "roofline": head["roofline"],
        "cpu_baseline": head.get("cpu_baseline"), "e2e": head["e2e"], "fp64_plain": head.get("fp64_plain"),
        "all_features": {k: allf[k] for k in ("value", "unit", "ms_per_step", "n_col", "class_limits_px",
                                               "class_limits_source", "phases_ms")},
        "configs": subs,
        "clocks": clk.summary(),
        "gpu_launches": head["gpu_launches"],
        "kernel_source": kernel_source_hash(),
    }
    print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
