"""Error of every output column of the CUDA path against the FP64 oracle.

Runs each benchmark workload through the library (the launch configuration
the benchmark times), computes the same ROIs with the oracle, and prints one
markdown table: per feature (direction-mean GLCM columns stand for their
per-offset columns), the largest relative error |gpu - oracle| / |oracle|
over the ROIs of each workload, and the largest error in units of the
parity tolerance of tests/parity_util.py (1.0 = at the tolerance).

    python tests/error_table.py [--configs blobs2d,nuclei2d,...] [--out FILE]

Needs a CUDA device.  The oracle runs on all host cores; the mosaic is
checked on a sample of its ROIs.
"""
from __future__ import annotations

import argparse
import os
import re
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path[:0] = [ROOT, HERE]

import oracle  # noqa: E402
from parity_util import EXACT, RTOL_GLCM, RTOL_STAT, scales  # noqa: E402

CONFIGS = ["blobs2d", "nuclei2d", "ct3d", "blobbatch", "mosaic_small"]
LABELS = {"blobs2d": "C1 (FP64 path)", "nuclei2d": "C2", "ct3d": "C3", "blobbatch": "C4",
          "mosaic_small": "C5 sample (8192² mosaic)"}


def _workload(name):
    from paper_2603_12016_gb300 import workloads as W

    if name == "mosaic_small":
        return W.mosaic_2d(size=8192, n_roi=32_000)
    return W.config(name)


def _gpu_and_oracle(name, sample, threads):
    import torch

    from paper_2603_12016_gb300 import nyx

    w = _workload(name)
    prm = w.params
    if name == "mosaic_small":
        img, mask = w.assemble()
        ndim = 2
    else:
        img, mask, ndim = w.image, w.mask, w.ndim
    tdt = {np.uint16: torch.uint16, np.int16: torch.int16, np.float32: torch.float32}[img.dtype.type]
    n_roi = int(sum(len(np.unique(m[m > 0])) for m in (mask.reshape((-1,) + mask.shape[-ndim:]))))
    ex = nyx.Extractor(img.shape, tdt, ndim=ndim, glcm_levels=prm.get("glcm_levels", 0) or 0,
                       dists=prm.get("dists", (1,)), glcm_per_offset_cols=(name == "blobs2d"),
                       hist_bins=prm.get("hist_bins", 256), precision="fp64" if name == "blobs2d" else "fp32",
                       max_rois=max(1024, 2 * n_roi))
    table = ex(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda()).cpu().numpy()
    g = {c: table[:, i] for i, c in enumerate(ex.columns)}
    keys = (g["IMAGE"].astype(np.int64) << 32) | g["LABEL"].astype(np.int64)
    rois = None
    if sample and len(keys) > sample:
        rng = np.random.default_rng(17)
        rois = sorted(int(k) for k in rng.choice(keys, size=sample, replace=False))
        sel = np.isin(keys, np.array(rois, dtype=np.int64))
        g = {k: v[sel] for k, v in g.items()}
    o = oracle.extract(img, mask, ndim, ng=max(prm.get("glcm_levels", 2) or 2, 2), dists=prm.get("dists", (1,)),
                       hist_bins=prm.get("hist_bins", 256), rois=rois, threads=threads, families=("glrlm", "glszm"))
    return g, o, ndim, len(g["LABEL"])


def _base(name):
    return re.sub(r"_D\d+(_A\d+|_O\d+)?$", "", name)


def errors(g, o, ndim):
    """{base feature: (max relative error, max error / tolerance)}"""
    out = {}
    for name, gv in g.items():
        if name not in o:
            continue
        ov = o[name]
        ok = ~(np.isnan(gv) & np.isnan(ov))
        if name in EXACT:
            rel = 0.0 if np.array_equal(gv[ok], ov[ok]) else float("inf")
            ratio = rel
        else:
            d = np.abs(gv - ov)
            with np.errstate(divide="ignore", invalid="ignore"):
                r = np.where(np.abs(ov) > 0, d / np.abs(ov), np.where(d == 0, 0.0, np.inf))
            rtol = RTOL_GLCM if name.startswith("GLCM_") else RTOL_STAT
            tol = rtol * np.maximum(np.abs(ov), scales(o, name, ndim))
            with np.errstate(divide="ignore", invalid="ignore"):
                q = np.where(tol > 0, d / tol, np.where(d == 0, 0.0, np.inf))
            rel = float(np.nanmax(r[ok])) if ok.any() else 0.0
            ratio = float(np.nanmax(q[ok])) if ok.any() else 0.0
        b = _base(name)
        pr, pq = out.get(b, (0.0, 0.0))
        out[b] = (max(pr, rel), max(pq, ratio))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", default=",".join(CONFIGS))
    ap.add_argument("--sample", type=int, default=600, help="ROIs per workload checked (0: all)")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    from paper_2603_12016_gb300 import build

    build.build()
    cols, res = [], {}
    for name in a.configs.split(","):
        t0 = time.time()
        g, o, ndim, n = _gpu_and_oracle(name, 0 if name in ("blobs2d", "nuclei2d") else a.sample, a.threads)
        res[name] = errors(g, o, ndim)
        cols.append(f"{LABELS.get(name, name)}, {n} ROIs")
        print(f"{name}: {n} ROIs compared in {time.time() - t0:.1f} s", file=sys.stderr)
    feats = sorted({f for r in res.values() for f in r})
    lines = ["| feature | " + " | ".join(cols) + " |", "|---|" + "---|" * len(cols)]
    for f in feats:
        cells = []
        for name in a.configs.split(","):
            if f not in res[name]:
                cells.append("—")
                continue
            rel, q = res[name][f]
            cells.append("exact" if rel == 0 and q == 0 else f"{rel:.1e} ({q:.2f})")
        lines.append(f"| {f} | " + " | ".join(cells) + " |")
    text = "\n".join(lines)
    print(text)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text + "\n")


if __name__ == "__main__":
    main()
