"""Plain FP64 CPU oracle for batched per-ROI feature extraction.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package.

The arithmetic lives in ``nyx_oracle.c`` (literal FP64 definitions, see the
header of that file for the paper passages each part follows); this module
only compiles it with gcc and marshals NumPy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nyx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DTYPE_CODES = {np.dtype(np.uint16): 0, np.dtype(np.int16): 1, np.dtype(np.float32): 2, np.dtype(np.float64): 3}
NAME_LEN = 48


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("batch", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("ng", ctypes.c_int),
        ("n_dist", ctypes.c_int),
        ("dist", ctypes.c_int * 8),
        ("hist_bins", ctypes.c_int),
        ("families", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        _lib.orc_n_features.argtypes = [P(OrcCfg)]
        _lib.orc_n_features.restype = ctypes.c_int
        _lib.orc_feature_names.argtypes = [P(OrcCfg), ctypes.c_char_p]
        _lib.orc_feature_names.restype = ctypes.c_int
        _lib.orc_count_rois.argtypes = [P(OrcCfg), ctypes.c_void_p]
        _lib.orc_count_rois.restype = ctypes.c_int64
        _lib.orc_extract.argtypes = [P(OrcCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        _lib.orc_extract.restype = ctypes.c_int64
        _lib.orc_roi_bins.argtypes = [P(OrcCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_int64]
        _lib.orc_roi_bins.restype = ctypes.c_int64
        _lib.orc_roi_glcm.argtypes = [P(OrcCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_void_p]
        _lib.orc_roi_glcm.restype = ctypes.c_int
        _lib.orc_glcm_features.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib.orc_glcm_features.restype = None
        _lib.orc_grad.argtypes = [P(OrcCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.orc_grad.restype = ctypes.c_int64
        _lib.orc_unit_dir.argtypes = [P(OrcCfg), ctypes.c_int, ctypes.c_void_p]
        _lib.orc_unit_dir.restype = None
    return _lib


GLCM_NAMES = ["ASM", "ACOR", "CLUPROM", "CLUSHADE", "CLUTEND", "CONTRAST", "CORR", "DIFAVE", "DIFENTRO", "DIFVAR",
              "DIS", "ENERGY", "ENTROPY", "HOM1", "HOM2", "IDM", "INFOMEAS1", "INFOMEAS2", "IDMN", "ID", "IDN", "IV",
              "JAVE", "JE", "JMAX", "SUMAVE", "SUMENT", "JVAR", "SUMVAR", "VARIANCE"]


FAMILIES = {"glrlm": 1, "glszm": 2}


def make_cfg(img: np.ndarray, ndim: int, ng: int = 0, dists: Sequence[int] = (1,), hist_bins: int = 256,
             families: Sequence[str] = ()) -> OrcCfg:
    """img: [batch,] [z,] y, x array.  ndim = 2 or 3 (spatial dims).
    families: optional texture families ("glrlm", "glszm") beyond the ones
    always computed; they need ng > 0."""
    shape = img.shape
    if ndim == 2:
        if img.ndim == 2:
            batch, nz, ny, nx = 1, 1, shape[0], shape[1]
        else:
            batch, nz, ny, nx = shape[0], 1, shape[1], shape[2]
    else:
        if img.ndim == 3:
            batch, nz, ny, nx = 1, shape[0], shape[1], shape[2]
        else:
            batch, nz, ny, nx = shape
    c = OrcCfg()
    c.ndim = ndim
    c.nx, c.ny, c.nz = nx, ny, nz
    c.batch = batch
    c.dtype = DTYPE_CODES[img.dtype]
    c.ng = ng
    c.n_dist = len(dists)
    for i, d in enumerate(dists):
        c.dist[i] = int(d)
    c.hist_bins = hist_bins
    c.families = sum(FAMILIES[f] for f in set(families))
    return c


def feature_names(cfg: OrcCfg) -> list:
    n = lib().orc_n_features(ctypes.byref(cfg))
    buf = ctypes.create_string_buffer(n * NAME_LEN)
    lib().orc_feature_names(ctypes.byref(cfg), buf)
    raw = buf.raw
    return [raw[i * NAME_LEN:(i + 1) * NAME_LEN].split(b"\0", 1)[0].decode() for i in range(n)]


def roi_key(image: int, label: int) -> int:
    return (int(image) << 32) | int(label)


def extract(img: np.ndarray, mask: np.ndarray, ndim: int, ng: int = 0, dists: Sequence[int] = (1,),
            hist_bins: int = 256, rois: Optional[Iterable[int]] = None, threads: int = 1,
            families: Sequence[str] = ()) -> Dict[str, np.ndarray]:
    """Compute every feature of every ROI (or of the ROI keys in ``rois``,
    key = image << 32 | label), plus the optional texture ``families``
    ("glrlm", "glszm").  Returns {feature name: FP64 array [n_roi]} in
    ascending key order."""
    img = np.ascontiguousarray(img)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    assert img.shape == mask.shape
    cfg = make_cfg(img, ndim, ng, dists, hist_bins, families)
    names = feature_names(cfg)
    if rois is not None:
        sub = np.ascontiguousarray(np.array(sorted(set(int(r) for r in rois)), dtype=np.int64))
        cap = len(sub)
        sub_ptr, n_sub = sub.ctypes.data, len(sub)
    else:
        n = lib().orc_count_rois(ctypes.byref(cfg), mask.ctypes.data)
        if n < 0:
            raise ValueError("oracle: negative label in mask")
        cap, sub_ptr, n_sub = n, None, 0
    out = np.zeros((max(cap, 1), len(names)), dtype=np.float64)
    got = lib().orc_extract(ctypes.byref(cfg), img.ctypes.data, mask.ctypes.data, sub_ptr, n_sub, cap,
                            out.ctypes.data, int(threads))
    if got < 0:
        raise ValueError(f"oracle: extract failed ({got})")
    out = out[:got]
    return {nm: out[:, i].copy() for i, nm in enumerate(names)}


def roi_bins(img, mask, ndim, key, nbins):
    img = np.ascontiguousarray(img)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    cfg = make_cfg(img, ndim)
    out = np.zeros(mask.size, dtype=np.int32)
    n = lib().orc_roi_bins(ctypes.byref(cfg), img.ctypes.data, mask.ctypes.data, int(key), int(nbins),
                           out.ctypes.data, out.size)
    if n < 0:
        raise KeyError(key)
    return out[:n]


def roi_glcm(img, mask, ndim, key, ng, direction, dist):
    img = np.ascontiguousarray(img)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    cfg = make_cfg(img, ndim, ng, (dist,))
    out = np.zeros((ng, ng), dtype=np.float64)
    if lib().orc_roi_glcm(ctypes.byref(cfg), img.ctypes.data, mask.ctypes.data, int(key), int(direction), int(dist),
                          out.ctypes.data) != 0:
        raise KeyError(key)
    return out


def glcm_features(P: np.ndarray) -> Dict[str, float]:
    P = np.ascontiguousarray(P, dtype=np.float64)
    ng = P.shape[0]
    out = np.zeros(30, dtype=np.float64)
    lib().orc_glcm_features(ng, P.ctypes.data, out.ctypes.data)
    return dict(zip(GLCM_NAMES, out.tolist()))


def unit_dir(ndim: int, k: int):
    cfg = OrcCfg()
    cfg.ndim = ndim
    out = np.zeros(3, dtype=np.int32)
    lib().orc_unit_dir(ctypes.byref(cfg), int(k), out.ctypes.data)
    return tuple(int(v) for v in out)


def grad(img: np.ndarray, mask: np.ndarray, ndim: int, gtab: Dict[str, np.ndarray]) -> np.ndarray:
    """dL/dI for L = sum over ROIs and features of gtab[name][roi] * feature;
    ``gtab`` maps feature names to per-ROI upstream gradients (ascending key
    order, missing names = 0).  Returns an FP64 array shaped like img."""
    img = np.ascontiguousarray(img)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    cfg = make_cfg(img, ndim, 0, (1,))
    names = feature_names(cfg)
    n = lib().orc_count_rois(ctypes.byref(cfg), mask.ctypes.data)
    g = np.zeros((max(n, 1), len(names)), dtype=np.float64)
    for i, nm in enumerate(names):
        if nm in gtab:
            g[:n, i] = gtab[nm]
    out = np.zeros(img.shape, dtype=np.float64)
    got = lib().orc_grad(ctypes.byref(cfg), img.ctypes.data, mask.ctypes.data, g.ctypes.data, out.ctypes.data)
    if got < 0:
        raise ValueError("oracle: grad failed")
    return out
