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
    """nvidia-smi samples (SM clock, max clock, throttle reasons) while the
    timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# DRAM bytes (read + write) per launch of a phase's kernel from one ncu
# capture (profiles/roi_kernels_nuclei2d_2048.md), keyed by workload, phase
# and class limits; entries are removed when the kernel changes.
TRAFFIC = {
    ("nuclei2d_2048_u16_4000roi", "roi_warp", (256, 1024, 8192)): 5.88e6,
    ("nuclei2d_2048_u16_4000roi", "roi_small", (256, 1024, 8192)): 16.58e6,
    ("nuclei2d_2048_u16_4000roi", "roi_medium", (256, 1024, 8192)): 13.68e6,
}


def roi_classes(w, lim_pix=None):
    """Pixels and ROI count per size class (warp, small, medium, multi-block)
    by the library's class rule: pixel count against the class limits
    (default 256 / 1,024 / 8,192) and padded bounding-box cells against the
    class capacities 1,024 / 4,096 / 16,384."""
    import numpy as np
    from scipy import ndimage

    pad = max(w.params["dists"]) if w.params["glcm_levels"] > 0 else 0
    lp = tuple(lim_pix) if lim_pix else (256, 1024, 8192)
    lims = ((lp[0], 1024), (lp[1], 4096), (lp[2], 16384))
    px, rows = [0, 0, 0, 0], [0, 0, 0, 0]
    masks = w.mask if (w.mask.ndim == 3 and w.ndim == 2) else w.mask[None]
    for m in masks:
        cnt = np.bincount(m.ravel())
        for lab, sl in enumerate(ndimage.find_objects(m), start=1):
            if sl is None:
                continue
            ext = [s.stop - s.start + 2 * pad for s in sl]
            cells = int(np.prod(ext))
            n = int(cnt[lab])
            k = 3
            for i in (2, 1, 0):
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


def make_workload(name: str, rank: int):
    from paper_2603_12016_gb300 import workloads as W

    if name.startswith("mosaic"):
        # whole-slide stand-in generated tile by tile; the assembled arrays are
        # what the host would stream
        big = name == "mosaic"
        m = W.mosaic_2d(size=32768 if big else 8192, tile=4096 if big else 1024,
                        n_roi=500_000 if big else 32_000, seed=1005 + rank)
        img, mask = m.assemble()
        n_roi = int(np.count_nonzero(np.bincount(mask.ravel())[1:]))
        return W.Workload(m.name, img, mask, 2, params=dict(m.params),
                          meta={"n_roi": n_roi, "tile": m.tile_size})
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
    labels = np.unique(mask[mask > 0])
    sample = labels[: min(len(labels), args.ref_rois)]
    keys = [oracle.roi_key(0, int(l)) for l in sample]
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


def _oracle_view(w):
    """Arrays the oracle samples from: the first 4096 x 4096 tile of a
    streamed mosaic (the oracle separates every pixel of its input first),
    else the whole workload."""
    if w.meta.get("tile"):
        return w.image[:4096, :4096], w.mask[:4096, :4096], " (first 4096x4096 tile)"
    return w.image, w.mask, ""


def cpu_baseline(w, budget_s: float):
    """Time the oracle on the host cores on a bounded ROI sample."""
    import numpy as np
    import oracle

    cores = os.cpu_count() or 1
    image, mask, where = _oracle_view(w)
    labels = np.unique(mask[mask > 0])
    prm = w.params
    n = 32
    while True:
        sample = labels[: min(n, len(labels))]
        keys = [oracle.roi_key(0, int(l)) for l in sample]
        t0 = time.perf_counter()
        oracle.extract(image, mask, w.ndim, ng=prm["glcm_levels"], dists=prm["dists"],
                       hist_bins=prm["hist_bins"], rois=keys, threads=cores)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or len(sample) == len(labels):
            break
        n = int(n * min(8.0, max(2.0, budget_s / 4 / max(dt, 1e-3))))
    return {"value": len(sample) / dt, "unit": "ROIs/s", "cores": cores, "kind": "oracle",
            "sample": f"first {len(sample)} of {len(labels)} ROIs of {w.name}{where}, {dt:.1f} s",
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
    """Device ms of one extraction of the workload with the NGTDM and GLDM
    families removed from the full feature set and alone."""
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


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nuclei2d")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison path")
    ap.add_argument("--ref-rois", type=int, default=800)
    ap.add_argument("--backward", dest="backward", action="store_true", default=None,
                    help="time forward + backward (default for the blobbatch workloads)")
    ap.add_argument("--no-backward", dest="backward", action="store_false")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default class limits")
    ap.add_argument("--class-limits", default=None, help="warp,small,medium pixel limits instead of autotuning")
    ap.add_argument("--sweep", default=None, choices=["soft", "scalability", "families"],
                    help="soft: the GLCM timing grid of Eqs. 2-5 on the 2048^2 nuclei workload and the Eq. 8 "
                         "separability grid on labelled texture classes; scalability: time over ROI size x ROI "
                         "count (GPU device, GPU end to end, CPU oracle) and the feature-group cost of an image "
                         "of 100 ROIs of 100,000 px; families: the workload with the NGTDM and GLDM removed "
                         "and alone (one JSON line each, not bench lines)")
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

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    from paper_2603_12016_gb300 import build, nyx

    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()

    w = make_workload(args.workload, rank)
    prm = w.params
    dtype = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[w.image.dtype.type]
    max_rois = 8192 if w.meta["n_roi"] <= 8192 else 2 * w.meta["n_roi"]
    tile = w.meta.get("tile")  # streamed mosaic: e2e goes through nyx_extract_tiles

    def extractor(precision):
        return nyx.Extractor(w.image.shape, dtype, ndim=w.ndim, glcm_levels=prm["glcm_levels"], dists=prm["dists"],
                             hist_bins=prm["hist_bins"], precision=precision, max_rois=max_rois, device=dev)

    ex = extractor("fp32")
    img = torch.from_numpy(w.image).to(dev)
    mask = torch.from_numpy(w.mask).to(dev)
    table = torch.empty((max_rois, len(ex.columns)), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # differentiation workload: a step is the forward pass plus the backward
    # pass for a fixed random upstream gradient dL/dtable
    bwd = args.backward if args.backward is not None else args.workload.startswith("blobbatch")
    gen = torch.Generator(device=dev).manual_seed(5)
    gtab = torch.randn((max_rois, len(ex.columns)), dtype=torch.float64, device=dev, generator=gen) if bwd else None
    gimg = torch.empty(img.shape, dtype=torch.float32, device=dev) if bwd else None

    def one_step(e, im, mk):
        n = e.extract_into(im, mk, table, save_for_backward=bwd)
        if bwd:
            e.backward(im, mk, gtab, out=gimg)
        return n

    def timed(e, steps, warmup):
        """Per-step device times (CUDA events on the launching stream) of
        back-to-back steps; the extraction replays its captured CUDA graph."""
        for _ in range(warmup):
            one_step(e, img, mask)
        e.sync_status()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for i in range(steps):
            flush.zero_()
            starts[i].record(stream)
            n = one_step(e, img, mask)
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        e.sync_status()
        return [s.elapsed_time(t) for s, t in zip(starts, ends)], int(n.item())

    def phase_profile(e, steps):
        """Per-phase times from the library's event ring (direct launches)."""
        e.profile(steps)
        for _ in range(steps):
            flush.zero_()
            one_step(e, img, mask)
        torch.cuda.synchronize(dev)
        e.sync_status()
        per = [e.phase_times(back=b) for b in range(steps)]
        e.profile(0)
        return {k: sum(p[k] for p in per) / steps for k in PHASES}

    limits = None
    if args.class_limits:
        limits = tuple(int(v) for v in args.class_limits.split(","))
        ex.set_class_limits(*limits)
    elif not args.no_autotune:
        limits = ex.autotune(img, mask, reps=3)
    with ClockSampler(local) as clk:
        ms, n_roi = timed(ex, args.steps, args.warmup)
    clocks = clk.summary()
    phases = phase_profile(ex, min(args.steps, 10))
    t_step, n_total = reduce_over_ranks(dist, dev, statistics.median(ms), n_roi)
    value = n_total / (t_step * 1e-3)
    px_total = w.image.size * world
    n_col = len(ex.columns)
    peak, peak_kind = _peaks()
    alg = algorithmic_bytes(w, n_roi, n_col)
    pipe_gbs = alg / (t_step * 1e-3) / 1e9

    # dominant kernel and its roofline: algorithmic bytes of the phase that
    # takes longest (the scan streams image + mask once; a ROI class reads
    # its ROIs' pixels and mask once and writes their table rows; the GLCM
    # feature kernel reads the per-offset sums and writes the GLCM columns)
    dom = max(phases, key=phases.get)
    cls_px, cls_rows = roi_classes(w, limits)
    n_off = len(prm["dists"]) * (13 if w.ndim == 3 else 4) if prm["glcm_levels"] > 0 else 0
    per_px = w.image.itemsize + 4
    dom_bytes = {"scan": w.image.nbytes + w.mask.nbytes,
                 "roi_warp": cls_px[0] * per_px + 8 * cls_rows[0] * n_col,
                 "roi_small": cls_px[1] * per_px + 8 * cls_rows[1] * n_col,
                 "roi_medium": cls_px[2] * per_px + 8 * cls_rows[2] * n_col,
                 "roi_big": cls_px[3] * per_px + 8 * cls_rows[3] * n_col,
                 "final": n_roi * (512 + n_off * 160 + 8 * n_col)}.get(dom, 0)
    dom_gbs = dom_bytes / (phases[dom] * 1e-3) / 1e9
    traffic = TRAFFIC.get((w.name, dom, tuple(limits) if limits else None))
    roofline = {"bound": "hbm", "kernel": dom, "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                "frac": dom_gbs / peak, "traffic": traffic, "peak_kind": peak_kind,
                "algorithmic_bytes": int(dom_bytes)}

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
        s, t = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        if tile is None:
            d_img.copy_(h_img, non_blocking=True)
            d_mask.copy_(h_mask, non_blocking=True)
            n = one_step(ex, d_img, d_mask)
        else:  # tiles streamed from host memory, band scans overlapping the host
            ex.extract_tiles(tile_source, (tile, tile), d_img, d_mask, table=table)
        h_table[:n_roi].copy_(table[:n_roi], non_blocking=True)
        if bwd:
            h_grad.copy_(gimg, non_blocking=True)
        t.record(stream)
        t.synchronize()
        if i >= args.warmup:
            e2e_ms.append(s.elapsed_time(t))
    e2e_t, _ = reduce_over_ranks(dist, dev, statistics.median(e2e_ms), n_roi)
    e2e = {"value": n_total / (e2e_t * 1e-3), "unit": "ROIs/s",
           "h2d_bytes_per_step": int(w.image.nbytes + w.mask.nbytes), "api": "nyx_extract_tiles" if tile else "nyx_extract",
           "d2h_bytes_per_step": int(8 * n_roi * n_col + (4 * w.image.size if bwd else 0)), "ms_per_step": e2e_t}

    fp64 = None
    if not args.no_fp64:
        ex64 = extractor("fp64")
        if limits is not None:
            ex64.set_class_limits(*limits)
        ms64, _ = timed(ex64, max(3, args.steps // 4), 3)
        t64 = statistics.median(ms64)
        fp64 = {"value": n_roi / (t64 * 1e-3), "unit": "ROIs/s", "ms_per_step": t64,
                "speedup_fp32_over_fp64": t64 / t_step}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, 20.0)
    # begin, scan, key sort, setup, the block classes whose pixel limit is
    # above 0, reset; multi-block class: zero, pass 1, pass 2, sorted order
    # statistics (+ GLCM, + NGTDM); statistics final (+ GLCM features)
    glcm = w.params["glcm_levels"] > 0
    n_cls = sum(1 for v in (limits or (256, 1024, 8192)) if v > 0)
    launches_per_step = 5 + n_cls + 4 + (2 if glcm else 0) + 1 + (1 if glcm else 0)
    if bwd:  # begin, scan, key sort, setup, coefficients, per-pixel gradient, reset
        launches_per_step += 7
    line = {
        "metric": METRIC, "value": value, "unit": "ROIs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
        "config": {"workload": w.name, "image": list(w.image.shape), "pixel_dtype": str(w.image.dtype),
                   "n_roi": n_roi, "n_col": n_col, "glcm_levels": prm["glcm_levels"], "dists": list(prm["dists"]),
                   "hist_bins": prm["hist_bins"], "features": "all", "step": "forward + backward" if bwd else "forward",
                   "l2": "flushed (256 MB write) between steps", "class_limits_px": list(limits) if limits else None,
                   "timing": "median of per-step CUDA-event times, CUDA-graph replay",
                   "parallelism": f"replicas{world}"},
        "mpix_per_s": px_total / (t_step * 1e-3) / 1e6,
        "roi_mpix_per_s": float((w.mask > 0).sum()) * world / (t_step * 1e-3) / 1e6,
        "pipeline_hbm": {"algorithmic_bytes": alg, "achieved_gbs": pipe_gbs, "frac": pipe_gbs / peak,
                         "peak": peak, "peak_kind": peak_kind},
        "phases_ms": phases,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fp64_plain": fp64,
        "clocks": clocks,
        "gpu_launches": launches_per_step * args.steps,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
