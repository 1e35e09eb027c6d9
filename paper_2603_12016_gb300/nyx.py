"""Python binding of libnyxgpu (the C ABI in include/nyx.h).

Argument marshalling only: every step of the extraction and of its backward
pass runs in the library's CUDA kernels.  PyTorch provides device memory,
the current stream and autograd.  There is no CPU path: if the library is
missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnyxgpu.so")

NYX_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_DTYPE", 3: "ERR_SHAPE", 4: "ERR_BAD_LABEL", 5: "ERR_NONFINITE",
                6: "ERR_CAPACITY", 7: "ERR_CUDA", 8: "ERR_OOM", 9: "ERR_TIMEOUT", 10: "ERR_STATE"}
DTYPES = {torch.uint16: 0, torch.int16: 1, torch.float32: 2}
SAVE_FOR_BACKWARD = 1
SYNC = 2


class NyxParams(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("ndim", ctypes.c_int32),
        ("dims", ctypes.c_int64 * 3),
        ("batch", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("feature_mask", ctypes.c_uint64 * 4),
        ("glcm_levels", ctypes.c_int32),
        ("n_dist", ctypes.c_int32),
        ("dists", ctypes.c_int32 * 8),
        ("glcm_per_offset_cols", ctypes.c_int32),
        ("hist_bins", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("max_rois", ctypes.c_int64),
    ]


class NyxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nyx {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


# int (*)(void* user, int64 x0, int64 y0, int64 w, int64 h, void* h_img, int32* h_mask)
TILE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p)


def lib() -> ctypes.CDLL:
    """Load libnyxgpu.so (built in-tree by build.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2603_12016_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, P = ctypes.c_void_p, ctypes.POINTER
    L.nyx_params_default.argtypes = [P(NyxParams), ctypes.c_int64, ctypes.c_int64]
    L.nyx_create.argtypes = [P(vp), ctypes.c_int]
    L.nyx_destroy.argtypes = [vp]
    L.nyx_destroy.restype = None
    L.nyx_last_error.argtypes = [vp]
    L.nyx_last_error.restype = ctypes.c_char_p
    L.nyx_plan_create.argtypes = [vp, P(NyxParams), P(vp)]
    L.nyx_plan_destroy.argtypes = [vp]
    L.nyx_plan_destroy.restype = None
    L.nyx_num_columns.argtypes = [vp, P(ctypes.c_int)]
    L.nyx_column_name.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]
    L.nyx_feature_id.argtypes = [ctypes.c_char_p]
    L.nyx_feature_id.restype = ctypes.c_int
    L.nyx_count_rois.argtypes = [vp, vp, vp, P(ctypes.c_int64), vp]
    L.nyx_extract.argtypes = [vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.c_uint32, vp]
    L.nyx_sync_status.argtypes = [vp, vp]
    L.nyx_backward.argtypes = [vp, vp, vp, vp, vp, vp]
    L.nyx_debug_select.argtypes = [vp, ctypes.c_int64]
    L.nyx_debug_glcm.argtypes = [vp, ctypes.c_int, vp]
    L.nyx_debug_bins.argtypes = [vp, vp, vp, vp, vp]
    L.nyx_count_rois_noalloc.argtypes = [P(NyxParams), vp, vp, P(ctypes.c_int64), vp]
    L.nyx_count_rois_noalloc.restype = ctypes.c_int
    L.nyx_profile_enable.argtypes = [vp, ctypes.c_int]
    L.nyx_phase_times.argtypes = [vp, ctypes.c_int, P(ctypes.c_float), ctypes.c_int]
    L.nyx_graph_phase_events.argtypes = [vp, ctypes.c_int]
    L.nyx_graph_phase_times.argtypes = [vp, P(ctypes.c_float), ctypes.c_int]
    L.nyx_extract_tiles.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, TILE_FN, vp, vp, vp, vp, ctypes.c_int64, vp,
                                    ctypes.c_uint32, vp]
    L.nyx_extract_tiles.restype = ctypes.c_int
    L.nyx_use_graphs.argtypes = [vp, ctypes.c_int]
    L.nyx_graph_captures.argtypes = [vp, P(ctypes.c_int64)]
    L.nyx_set_class_limits.argtypes = [vp, P(ctypes.c_int32)]
    L.nyx_autotune.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int, vp, P(ctypes.c_int32)]
    L.nyx_set_tuning.argtypes = [vp, P(ctypes.c_int32)]
    L.nyx_get_tuning.argtypes = [vp, P(ctypes.c_int32)]
    L.nyx_set_scan_staging.argtypes = [vp, ctypes.c_int]
    L.nyx_get_scan_staging.argtypes = [vp, P(ctypes.c_int)]
    for f in ("nyx_params_default", "nyx_create", "nyx_plan_create", "nyx_num_columns", "nyx_column_name",
              "nyx_count_rois", "nyx_extract", "nyx_sync_status", "nyx_backward", "nyx_debug_select",
              "nyx_debug_glcm", "nyx_debug_bins", "nyx_profile_enable", "nyx_phase_times", "nyx_use_graphs",
              "nyx_graph_captures", "nyx_set_class_limits", "nyx_autotune", "nyx_graph_phase_events",
              "nyx_graph_phase_times", "nyx_set_tuning", "nyx_get_tuning", "nyx_set_scan_staging",
              "nyx_get_scan_staging"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def feature_id(name: str) -> int:
    return lib().nyx_feature_id(name.encode())


# Feature ids of the hot-path feature set: first-order and order statistics
# with the histogram features (Table S1 / S5, ids 0-40), raw / central /
# normalised moments with Hu invariants (Table S2 / S5, ids 41-50) and the
# GLCM features (Table S3, ids 51-80).  Ids 81 and up are the edge intensity
# statistics, NGTDM, GLDM, GLRLM and GLSZM.
CORE_FEATURE_IDS = tuple(range(81))


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Extractor:
    """A plan: fixed image shape, dtype and hyperparameters.

    shape: (H, W) / (B, H, W) for ndim=2, (D, H, W) / (B, D, H, W) for
    ndim=3.  features: iterable of feature names (see nyx_feature_id) or
    feature ids, or None for every feature (untargeted extraction)."""

    def __init__(self, shape: Sequence[int], dtype: torch.dtype, ndim: int = 2, glcm_levels: int = 64,
                 dists: Sequence[int] = (1,), glcm_per_offset_cols: bool = False, hist_bins: int = 256,
                 precision: str = "fp32", features: Optional[Iterable[str]] = None, max_rois: int = 65536,
                 device: Optional[torch.device] = None):
        L = lib()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        shape = tuple(int(s) for s in shape)
        spatial = shape[-ndim:]
        batch = 1
        for s in shape[:-ndim]:
            batch *= s
        self.shape, self.ndim, self.dtype = shape, ndim, dtype
        p = NyxParams()
        L.nyx_params_default(ctypes.byref(p), 1, 1)
        p.ndim = ndim
        p.dims[0] = spatial[-1]
        p.dims[1] = spatial[-2]
        p.dims[2] = spatial[0] if ndim == 3 else 1
        p.batch = batch
        if dtype not in DTYPES:
            raise NyxError(2, f"unsupported dtype {dtype}")
        p.dtype = DTYPES[dtype]
        if features is not None:
            mask = [0, 0, 0, 0]
            for f in features:
                fid = int(f) if isinstance(f, int) else feature_id(f)
                if fid < 0:
                    raise KeyError(f"unknown feature {f}")
                mask[fid >> 6] |= 1 << (fid & 63)
            for i in range(4):
                p.feature_mask[i] = mask[i]
        p.glcm_levels = glcm_levels
        p.n_dist = len(dists)
        for i, d in enumerate(dists):
            p.dists[i] = int(d)
        p.glcm_per_offset_cols = 1 if glcm_per_offset_cols else 0
        p.hist_bins = hist_bins
        p.precision = {"fp32": 0, "fp64": 1}[precision]
        p.max_rois = max_rois
        self.params = p
        self.max_rois = max_rois
        self._ctx = ctypes.c_void_p()
        self._check(L.nyx_create(ctypes.byref(self._ctx), self.device.index or 0), None)
        self._plan = ctypes.c_void_p()
        self._check(L.nyx_plan_create(self._ctx, ctypes.byref(p), ctypes.byref(self._plan)))
        n = ctypes.c_int()
        L.nyx_num_columns(self._plan, ctypes.byref(n))
        buf = ctypes.create_string_buffer(64)
        self.columns: List[str] = []
        for i in range(n.value):
            L.nyx_column_name(self._plan, i, buf, 64)
            self.columns.append(buf.value.decode())
        self._n_roi = torch.zeros(1, dtype=torch.int64, device=self.device)

    def _check(self, st: int, ctx="default"):
        if st != NYX_OK:
            msg = lib().nyx_last_error(self._ctx).decode() if ctx is not None and self._ctx else ""
            raise NyxError(st, msg)

    def __del__(self):
        try:
            L = lib()
            if getattr(self, "_plan", None):
                L.nyx_plan_destroy(self._plan)
            if getattr(self, "_ctx", None):
                L.nyx_destroy(self._ctx)
        except Exception:
            pass

    def _inputs(self, img: torch.Tensor, mask: torch.Tensor):
        if img.device.type != "cuda" or mask.device.type != "cuda":
            raise NyxError(1, "image and mask must be CUDA tensors")
        if tuple(img.shape) != self.shape or tuple(mask.shape) != self.shape:
            raise NyxError(3, f"expected shape {self.shape}, got {tuple(img.shape)} / {tuple(mask.shape)}")
        if img.dtype != self.dtype or mask.dtype != torch.int32:
            raise NyxError(2, "image dtype differs from the plan or mask is not int32")
        return img.contiguous(), mask.contiguous()

    def count_rois(self, img: torch.Tensor, mask: torch.Tensor) -> int:
        img, mask = self._inputs(img, mask)
        n = ctypes.c_int64()
        self._check(lib().nyx_count_rois(self._plan, img.data_ptr(), mask.data_ptr(), ctypes.byref(n),
                                         _stream_ptr(self.device)))
        return n.value

    def extract_into(self, img: torch.Tensor, mask: torch.Tensor, table: torch.Tensor, save_for_backward=False,
                     sync=False) -> torch.Tensor:
        """Asynchronous extraction into a preallocated FP64 [cap, n_col]
        table; returns the device int64 ROI count."""
        img, mask = self._inputs(img, mask)
        if table.dtype != torch.float64 or not table.is_contiguous() or table.dim() != 2 or \
                table.shape[1] != len(self.columns):
            raise NyxError(1, "table must be a contiguous float64 [cap, n_col] tensor")
        flags = (SAVE_FOR_BACKWARD if save_for_backward else 0) | (SYNC if sync else 0)
        self._check(lib().nyx_extract(self._plan, img.data_ptr(), mask.data_ptr(), table.data_ptr(), table.shape[0],
                                      self._n_roi.data_ptr(), flags, _stream_ptr(self.device)))
        return self._n_roi

    def __call__(self, img: torch.Tensor, mask: torch.Tensor, cap: Optional[int] = None,
                 save_for_backward: bool = False) -> torch.Tensor:
        """Extract and return the FP64 table [n_roi, n_col] (synchronises)."""
        cap = self.max_rois if cap is None else cap
        table = torch.empty((cap, len(self.columns)), dtype=torch.float64, device=self.device)
        n = self.extract_into(img, mask, table, save_for_backward=save_for_backward, sync=True)
        return table[: int(n.item())]

    def sync_status(self):
        self._check(lib().nyx_sync_status(self._plan, _stream_ptr(self.device)))

    def backward(self, img: torch.Tensor, mask: torch.Tensor, grad_table: torch.Tensor,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """dL/dimage (float32, image shape) of the last forward pass saved for
        backward, given dL/dtable (FP64 [rows, n_col]); asynchronous."""
        img, mask = self._inputs(img, mask)
        g = grad_table.to(dtype=torch.float64).contiguous()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        elif out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != tuple(self.shape):
            raise NyxError(1, "out must be a contiguous float32 tensor of the image shape")
        self._check(lib().nyx_backward(self._plan, img.data_ptr(), mask.data_ptr(), g.data_ptr(), out.data_ptr(),
                                       _stream_ptr(self.device)))
        return out

    PHASES = ("scan", "sort_setup", "roi_warp", "roi_small", "roi_medium", "roi_large", "roi_big", "final", "reset")
    N_CLASSES = 4  # block classes: warp, small, medium, large

    def extract_tiles(self, source, tile: Tuple[int, int], d_img: torch.Tensor, d_mask: torch.Tensor,
                      table: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Streamed extraction of a 2D mosaic: source(x0, y0, w, h) returns the
        (image, mask) numpy arrays of one tile; d_img / d_mask are the device
        buffers of the whole mosaic (filled here).  Returns the table rows."""
        import numpy as np

        img_dt = {torch.uint16: np.uint16, torch.int16: np.int16, torch.float32: np.float32}[self.dtype]
        err = []

        def cb(user, x0, y0, w, h, p_img, p_mask):
            try:
                ti, tm = source(int(x0), int(y0), int(w), int(h))
                ti = np.ascontiguousarray(ti, dtype=img_dt)
                tm = np.ascontiguousarray(tm, dtype=np.int32)
                if ti.shape != (h, w) or tm.shape != (h, w):
                    raise ValueError(f"tile ({x0},{y0}) has shape {ti.shape}/{tm.shape}, expected {(h, w)}")
                ctypes.memmove(p_img, ti.ctypes.data, ti.nbytes)
                ctypes.memmove(p_mask, tm.ctypes.data, tm.nbytes)
                return 0
            except Exception as e:  # reported after the call
                err.append(e)
                return 1

        fn = TILE_FN(cb)
        if table is None:
            table = torch.empty((self.max_rois, len(self.columns)), dtype=torch.float64, device=self.device)
        st = lib().nyx_extract_tiles(self._plan, int(tile[0]), int(tile[1]), fn, None, d_img.data_ptr(),
                                     d_mask.data_ptr(), table.data_ptr(), table.shape[0], self._n_roi.data_ptr(),
                                     SYNC, _stream_ptr(self.device))
        if err:
            raise err[0]
        self._check(st)
        return table[: int(self._n_roi.item())]

    def use_graphs(self, enable: bool = True):
        """Replay the extraction as a captured CUDA graph (default on)."""
        self._check(lib().nyx_use_graphs(self._plan, int(bool(enable))))

    def graph_captures(self) -> int:
        n = ctypes.c_int64(0)
        self._check(lib().nyx_graph_captures(self._plan, ctypes.byref(n)))
        return int(n.value)

    def set_class_limits(self, warp: int, small: int, medium: int, large: int):
        """Pixel limits of the warp / small / medium / large block classes (0
        disables one; capacities 256 / 1,024 / 4,096 / 8,192 px)."""
        lim = (ctypes.c_int32 * 4)(warp, small, medium, large)
        self._check(lib().nyx_set_class_limits(self._plan, lim))

    def autotune(self, img: torch.Tensor, mask: torch.Tensor, reps: int = 5) -> Tuple[int, ...]:
        """Time a grid of class limits, then of label-scan tile heights under
        both row stagings, on this input (L2 flushed before every timed
        call), keep the fastest; returns tuning()."""
        img, mask = self._inputs(img, mask)
        table = torch.empty((self.max_rois, len(self.columns)), dtype=torch.float64, device=self.device)
        lim = (ctypes.c_int32 * 4)()
        self._check(lib().nyx_autotune(self._plan, img.data_ptr(), mask.data_ptr(), table.data_ptr(), table.shape[0],
                                       int(reps), _stream_ptr(self.device), lim))
        return self.tuning()

    def tuning(self) -> Tuple[int, ...]:
        """(warp, small, medium, large pixel limits, scan rows per warp (0 =
        chosen per call), scan staging (0 = bulk tensor copies where the row
        pitch allows, 1 = register loads))."""
        t = (ctypes.c_int32 * 5)()
        self._check(lib().nyx_get_tuning(self._plan, t))
        g = ctypes.c_int(0)
        self._check(lib().nyx_get_scan_staging(self._plan, ctypes.byref(g)))
        return tuple(int(v) for v in t) + (int(g.value),)

    def set_tuning(self, warp: int, small: int, medium: int, large: int, scan_rows: int = 0, scan_staging: int = 0):
        t = (ctypes.c_int32 * 5)(warp, small, medium, large, scan_rows)
        self._check(lib().nyx_set_tuning(self._plan, t))
        self._check(lib().nyx_set_scan_staging(self._plan, int(scan_staging)))

    def set_scan_staging(self, mode: int):
        """Label-scan row staging: 0 = bulk tensor copies into shared memory
        where the row pitch allows (default), 1 = register loads."""
        self._check(lib().nyx_set_scan_staging(self._plan, int(mode)))

    def profile(self, slots: int = 1):
        """Record per-phase CUDA events for the next extracts (ring of
        `slots`; 0 = off)."""
        self._check(lib().nyx_profile_enable(self._plan, int(slots)))

    def phase_times(self, back: int = 0) -> dict:
        ms = (ctypes.c_float * len(self.PHASES))()
        self._check(lib().nyx_phase_times(self._plan, int(back), ms, len(self.PHASES)))
        return dict(zip(self.PHASES, [float(v) for v in ms]))

    GRAPH_PHASES = ("scan", "sort_setup", "roi_warp", "roi_small", "roi_medium", "roi_large", "roi_big",
                    "glcm_final", "stats_final", "reset", "roi_stage", "all", "roi_runzone")

    def graph_phase_events(self, enable: bool = True):
        """Record a begin and an end event around each phase inside the
        replayed CUDA graph, on the stream the phase runs on."""
        self._check(lib().nyx_graph_phase_events(self._plan, int(bool(enable))))

    def graph_phase_times(self) -> dict:
        """Per-phase durations (ms) of the most recent graph replay."""
        ms = (ctypes.c_float * len(self.GRAPH_PHASES))()
        self._check(lib().nyx_graph_phase_times(self._plan, ms, len(self.GRAPH_PHASES)))
        return dict(zip(self.GRAPH_PHASES, [float(v) for v in ms]))

    def debug_select(self, roi: int):
        self._check(lib().nyx_debug_select(self._plan, int(roi)))

    def debug_glcm(self, off: int):
        import numpy as np

        ng = self.params.glcm_levels
        out = np.zeros((ng, ng), dtype=np.uint32)
        self._check(lib().nyx_debug_glcm(self._plan, int(off), out.ctypes.data))
        return out

    def debug_bins(self, img: torch.Tensor, mask: torch.Tensor) -> torch.Tensor:
        img, mask = self._inputs(img, mask)
        out = torch.empty(self.shape, dtype=torch.uint16, device=self.device)
        self._check(lib().nyx_debug_bins(self._plan, img.data_ptr(), mask.data_ptr(), out.data_ptr(),
                                         _stream_ptr(self.device)))
        return out


class _FeatureFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, mask, ex: Extractor):
        table = ex(img.detach(), mask, save_for_backward=True)
        ctx.ex = ex
        ctx.save_for_backward(img, mask)
        ctx.n_roi = table.shape[0]
        return table

    @staticmethod
    def backward(ctx, grad_table):
        img, mask = ctx.saved_tensors
        g = torch.zeros((ctx.ex.max_rois, grad_table.shape[1]), dtype=torch.float64, device=grad_table.device)
        g[: ctx.n_roi] = grad_table
        return ctx.ex.backward(img.detach(), mask, g), None, None


class FeatureLayer(torch.nn.Module):
    """Per-ROI features as a differentiable layer: forward returns the FP64
    feature table [n_roi, n_col]; backward propagates to the float32 image
    through the smooth intensity features (nyx_backward)."""

    def __init__(self, shape, ndim: int = 2, **kw):
        super().__init__()
        kw.setdefault("glcm_levels", 0)
        self.ex = Extractor(shape, torch.float32, ndim=ndim, **kw)
        self.columns = self.ex.columns

    def forward(self, img: torch.Tensor, mask: torch.Tensor) -> torch.Tensor:
        return _FeatureFn.apply(img, mask, self.ex)


def extract(img: torch.Tensor, mask: torch.Tensor, ndim: Optional[int] = None, **kw) -> Tuple[torch.Tensor, List[str]]:
    """One-shot extraction: returns (table [n_roi, n_col] float64, column names)."""
    if ndim is None:
        if img.dim() == 3:
            raise ValueError("ndim is ambiguous for a 3-dimensional tensor; pass ndim=2 (batch) or ndim=3 (volume)")
        ndim = 2 if img.dim() == 2 else 3
    ex = Extractor(tuple(img.shape), img.dtype, ndim=ndim, device=img.device, **kw)
    return ex(img, mask), ex.columns
