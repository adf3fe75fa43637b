"""ctypes binding of libtmgb.so -- argument marshalling only.

The functions below carry the C ABI's names (``include/tmgb.h``); every step of the
indexing path runs in the library's CUDA kernels.  There is no CPU fallback: if the
shared library is missing or the GPU is not usable, calls raise ``TmError``.

``Context`` wraps the handle for PyTorch users: device memory and streams come from
``torch`` tensors and ``torch.cuda`` streams.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmgb.so")

TM_OK, TM_ERR_INVALID_ARG, TM_ERR_OOM, TM_ERR_CUDA, TM_ERR_TIMEOUT = 0, 1, 2, 3, 4
TM_ERR_BUSY, TM_ERR_CANCELLED, TM_ERR_NOT_FOUND, TM_ERR_UNSUPPORTED = 5, 6, 7, 8
TM_DTYPE_U16, TM_DTYPE_F32 = 0, 1
TM_COORDS_POLAR, TM_COORDS_XY = 0, 1
TM_LIB_MIRROR, TM_LIB_UNIT_INTENSITY = 1, 2
TM_PATH_FP32_SPARSE, TM_PATH_BF16_RESCORE = 0, 1
TM_INDEX_GRAPH = 1
TM_INDEX_TEST_STALL = 2
TM_INDEX_REFINE = 4


class TmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tmgb error {code}: {msg}")
        self.code = code


class tm_library_desc(ctypes.Structure):
    _fields_ = [("n_templates", ctypes.c_int64), ("spot_offsets", ctypes.c_void_p),
                ("spot_a", ctypes.c_void_p), ("spot_b", ctypes.c_void_p),
                ("intensity", ctypes.c_void_p), ("coords", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("px_per_unit", ctypes.c_double),
                ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("dr", ctypes.c_double)]


class tm_library_info(ctypes.Structure):
    _fields_ = [("n_templates", ctypes.c_int64), ("n_base", ctypes.c_int64),
                ("n_spots", ctypes.c_int64), ("max_spots", ctypes.c_int32),
                ("mirror", ctypes.c_int32), ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32),
                ("dr", ctypes.c_double), ("n_symmetric", ctypes.c_int64),
                ("macs_per_pattern", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class tm_index_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("subtract", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("prefilter_fraction", ctypes.c_double), ("top_n", ctypes.c_int32),
                ("path", ctypes.c_int32), ("rescore_k", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("pixel_mask", ctypes.c_void_p), ("threshold", ctypes.c_double)]


class tm_hit(ctypes.Structure):
    _fields_ = [("template_index", ctypes.c_int32), ("shift", ctypes.c_int32),
                ("score", ctypes.c_float), ("angle_deg", ctypes.c_float), ("mirror", ctypes.c_int32)]


class tm_stats(ctypes.Structure):
    _fields_ = [("patterns", ctypes.c_int64), ("correlations", ctypes.c_int64),
                ("templates_scored", ctypes.c_int64), ("launches", ctypes.c_int64)]


class tm_server_params(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("tile_patterns", ctypes.c_int32), ("max_H", ctypes.c_int32),
                ("max_W", ctypes.c_int32), ("max_libs", ctypes.c_int32), ("max_top_n", ctypes.c_int32),
                ("queue_bytes", ctypes.c_size_t), ("blocking_submit", ctypes.c_int32),
                ("priority_slots", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_size_t),
                ("reserve_sms", ctypes.c_int32)]


class tm_request(ctypes.Structure):
    _fields_ = [("frames_host", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("H", ctypes.c_int32),
                ("W", ctypes.c_int32), ("n", ctypes.c_int64), ("lib_ids", ctypes.c_void_p),
                ("n_libs", ctypes.c_int32), ("priority", ctypes.c_int32), ("params", tm_index_params),
                ("out_host", ctypes.c_void_p), ("frames_dev", ctypes.c_void_p)]


class tm_request_status(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("tiles", ctypes.c_int32), ("submit_ms", ctypes.c_double),
                ("first_dispatch_ms", ctypes.c_double), ("done_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("h2d_ms", ctypes.c_double), ("kernels_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double)]


TM_STAGE_COUNT = 8
STAGES = ["polar", "prefilter", "sparse", "dft", "dense", "rescore", "gemm", "select"]


class tm_preprocess_params(ctypes.Structure):
    _fields_ = [("dog_sigma_min", ctypes.c_double), ("dog_sigma_max", ctypes.c_double),
                ("blur_sigma", ctypes.c_double), ("truncate", ctypes.c_double)]


class tm_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * TM_STAGE_COUNT), ("launches", ctypes.c_int64 * TM_STAGE_COUNT),
                ("sparse_macs", ctypes.c_int64)]


HIT_DTYPE = np.dtype([("template_index", "<i4"), ("shift", "<i4"), ("score", "<f4"),
                      ("angle_deg", "<f4"), ("mirror", "<i4")])
assert HIT_DTYPE.itemsize == ctypes.sizeof(tm_hit) == 20

_P = ctypes.c_void_p
_SIGS = {
    "tm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "tm_destroy": (None, [_P]),
    "tm_last_error": (ctypes.c_char_p, []),
    "tm_load_library": (ctypes.c_int, [_P, ctypes.POINTER(tm_library_desc), ctypes.POINTER(ctypes.c_int)]),
    "tm_unload_library": (ctypes.c_int, [_P, ctypes.c_int]),
    "tm_library_info_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(tm_library_info)]),
    "tm_library_export": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]),
    "tm_library_prepare_host": (ctypes.c_int, [ctypes.POINTER(tm_library_desc), ctypes.POINTER(tm_library_info),
                                               _P, _P, _P, _P, _P, _P, _P, _P]),
    "tm_library_bound_entries_host": (ctypes.c_int, [ctypes.POINTER(tm_library_desc), ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.POINTER(ctypes.c_int64), _P, _P, _P]),
    "tm_polar_transform": (ctypes.c_int, [_P, ctypes.POINTER(tm_index_params), _P, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_double, _P, _P, _P, _P]),
    "tm_prefilter": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_double, _P, _P, _P]),
    "tm_correlate": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "tm_index_patterns": (ctypes.c_int, [_P, ctypes.POINTER(tm_index_params), _P, ctypes.c_int32, ctypes.c_int64,
                                         ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32, _P,
                                         ctypes.POINTER(tm_stats), _P]),
    "tm_index_patterns_host": (ctypes.c_int, [_P, ctypes.POINTER(tm_index_params), _P, ctypes.c_int32,
                                              ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32,
                                              _P, ctypes.c_int64, ctypes.POINTER(tm_stats)]),
    "tm_index_params_default": (None, [ctypes.POINTER(tm_index_params)]),
    "tm_find_centres": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _P, _P]),
    "tm_orientation_vectors": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int64,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P]),
    "tm_angular_deviation": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "tm_kinematic_spots": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int32, _P, _P, _P]),
    "tm_preprocess": (ctypes.c_int, [_P, ctypes.POINTER(tm_preprocess_params), _P, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "tm_frame_sum": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, _P, _P]),
    "tm_matrix_mask": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "tm_prescore": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int64, ctypes.c_double, _P, _P]),
    "tm_check": (ctypes.c_int, [_P, _P]),
    "tm_index_patterns_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(tm_index_params), _P, ctypes.c_int32,
                                                 ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                                 _P]),
    "tm_autotune": (ctypes.c_int, [_P, ctypes.POINTER(tm_index_params), _P, ctypes.c_int32, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                   _P]),
    "tm_server_params_default": (None, [ctypes.POINTER(tm_server_params)]),
    "tm_server_create": (ctypes.c_int, [_P, ctypes.POINTER(tm_server_params), ctypes.POINTER(_P)]),
    "tm_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(tm_request), ctypes.POINTER(ctypes.c_uint64)]),
    "tm_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(tm_request_status)]),
    "tm_server_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "tm_server_pause": (ctypes.c_int, [_P, ctypes.c_int32]),
    "tm_server_destroy": (None, [_P]),
    "tm_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "tm_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(tm_profile)]),
}

_LIB = None


def library(path: str | None = None):
    """Load libtmgb.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise TmError(TM_ERR_CUDA, f"{p} is missing; build it with paper_2111_07347_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(rc: int):
    if rc != TM_OK:
        raise TmError(rc, library().tm_last_error().decode(errors="replace"))


# ---------------------------------------------------------------- C ABI, same names

def tm_last_error() -> str:
    return library().tm_last_error().decode(errors="replace")


def tm_index_params_default() -> tm_index_params:
    p = tm_index_params()
    library().tm_index_params_default(ctypes.byref(p))
    return p


def tm_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = _P()
    _check(library().tm_create(device, hbm_budget_bytes, ctypes.byref(h)))
    return h.value


def tm_destroy(ctx: int) -> None:
    library().tm_destroy(ctx)


class _Desc:
    """Keeps the numpy arrays behind a tm_library_desc alive."""

    def __init__(self, ts, n_r, n_theta, dr, mirror, unit_intensity):
        self.off = np.ascontiguousarray(ts.offsets, dtype=np.int64)
        self.a = np.ascontiguousarray(ts.a, dtype=np.float64)
        self.b = np.ascontiguousarray(ts.b, dtype=np.float64)
        self.I = np.ascontiguousarray(ts.intensity, dtype=np.float64)
        mirror = ts.mirror if mirror is None else mirror
        d = tm_library_desc()
        d.n_templates = self.off.shape[0] - 1
        d.spot_offsets = self.off.ctypes.data
        d.spot_a = self.a.ctypes.data if self.a.size else None
        d.spot_b = self.b.ctypes.data if self.b.size else None
        d.intensity = self.I.ctypes.data if self.I.size else None
        d.coords = TM_COORDS_XY if ts.coords == "xy" else TM_COORDS_POLAR
        d.flags = (TM_LIB_MIRROR if mirror else 0) | (TM_LIB_UNIT_INTENSITY if unit_intensity else 0)
        d.px_per_unit = float(getattr(ts, "px_per_unit", 1.0))
        d.n_r, d.n_theta, d.dr = int(n_r), int(n_theta), float(dr)
        self.desc = d


def _info_dict(info: tm_library_info) -> dict:
    return {name: getattr(info, name) for name, _ in tm_library_info._fields_}


def tm_library_prepare_host(ts, n_r: int, n_theta: int, dr: float = 1.0, mirror=None,
                            unit_intensity: bool = False) -> dict:
    """Host-side library preparation (no GPU): rounded/merged templates as numpy arrays."""
    d = _Desc(ts, n_r, n_theta, dr, mirror, unit_intensity)
    info = tm_library_info()
    _check(library().tm_library_prepare_host(ctypes.byref(d.desc), ctypes.byref(info), None, None, None,
                                             None, None, None, None, None))
    out = _alloc_export(info)
    out["packed"] = np.zeros(info.n_spots, np.int32)
    out["packed2"] = np.zeros(info.n_spots, np.int32)
    _check(library().tm_library_prepare_host(ctypes.byref(d.desc), ctypes.byref(info), *_export_ptrs(out),
                                             out["packed"].ctypes.data if out["packed"].size else None,
                                             out["packed2"].ctypes.data if out["packed2"].size else None))
    out["info"] = _info_dict(info)
    return out


def tm_library_bound_entries_host(ts, n_r: int, n_theta: int, dr: float = 1.0, mirror=None,
                                  unit_intensity: bool = False) -> dict:
    """The sparse kernel's spot-count-ordered bound entries (no GPU): order, word_start,
    entries [n][2] int32."""
    d = _Desc(ts, n_r, n_theta, dr, mirror, unit_intensity)
    nw, ne = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(library().tm_library_bound_entries_host(ctypes.byref(d.desc), ctypes.byref(nw), ctypes.byref(ne),
                                                   None, None, None))
    out = dict(order=np.zeros(nw.value * 32, np.int32), word_start=np.zeros(nw.value, np.int32),
               entries=np.zeros((ne.value, 2), np.int32))
    _check(library().tm_library_bound_entries_host(ctypes.byref(d.desc), ctypes.byref(nw), ctypes.byref(ne),
                                                   out["order"].ctypes.data, out["word_start"].ctypes.data,
                                                   out["entries"].ctypes.data if ne.value else None))
    return out


def _alloc_export(info):
    K, S = info.n_templates, info.n_spots
    return dict(offsets=np.zeros(K + 1, np.int64), r=np.zeros(S, np.int32), t=np.zeros(S, np.int32),
                intensity=np.zeros(S, np.float32), norm=np.zeros(K, np.float32), order=np.zeros(K, np.int32))


def _export_ptrs(out):
    return [out[k].ctypes.data if out[k].size else None
            for k in ("offsets", "r", "t", "intensity", "norm", "order")]


def tm_load_library(ctx: int, ts, n_r: int, n_theta: int, dr: float = 1.0, mirror=None,
                    unit_intensity: bool = False) -> int:
    d = _Desc(ts, n_r, n_theta, dr, mirror, unit_intensity)
    lid = ctypes.c_int()
    _check(library().tm_load_library(ctx, ctypes.byref(d.desc), ctypes.byref(lid)))
    return lid.value


def tm_unload_library(ctx: int, lib_id: int) -> None:
    _check(library().tm_unload_library(ctx, lib_id))


def tm_library_info_get(ctx: int, lib_id: int) -> dict:
    info = tm_library_info()
    _check(library().tm_library_info_get(ctx, lib_id, ctypes.byref(info)))
    return _info_dict(info)


def tm_library_export(ctx: int, lib_id: int) -> dict:
    info = tm_library_info()
    _check(library().tm_library_info_get(ctx, lib_id, ctypes.byref(info)))
    out = _alloc_export(info)
    _check(library().tm_library_export(ctx, lib_id, *_export_ptrs(out)))
    out["info"] = _info_dict(info)
    return out


def make_params(gamma=0.5, subtract=0.0, cx=math.nan, cy=math.nan, prefilter=1.0, top_n=5,
                path=TM_PATH_FP32_SPARSE, rescore_k=256, mask=None, threshold=0.0) -> tm_index_params:
    """mask: device uint8 tensor [H][W] (pixels with 0 read as 0) or None; threshold > 0: raw
    pixels below it read as 0."""
    p = tm_index_params_default()
    p.gamma, p.subtract, p.cx, p.cy = gamma, subtract, cx, cy
    p.prefilter_fraction, p.top_n, p.path, p.rescore_k = prefilter, top_n, path, rescore_k
    p.pixel_mask = None if mask is None else mask.data_ptr()
    p.threshold = threshold
    return p


def tm_polar_transform(ctx, params, frames_ptr, dtype, n, H, W, centres_ptr, n_r, n_theta, dr, polar_ptr, norm_ptr,
                       radial_ptr, stream) -> None:
    _check(library().tm_polar_transform(ctx, ctypes.byref(params), frames_ptr, dtype, n, H, W, centres_ptr, n_r,
                                        n_theta, dr, polar_ptr, norm_ptr, radial_ptr, stream))


def tm_prefilter(ctx, lib_id, radial_ptr, n, fraction, mask_ptr, score_ptr, stream) -> None:
    _check(library().tm_prefilter(ctx, lib_id, radial_ptr, n, fraction, mask_ptr, score_ptr, stream))


def tm_correlate(ctx, lib_id, polar_ptr, norm_ptr, n, mask_ptr, q_ptr, s_ptr, stream) -> None:
    _check(library().tm_correlate(ctx, lib_id, polar_ptr, norm_ptr, n, mask_ptr, q_ptr, s_ptr, stream))


def tm_prescore(ctx, lib_id, polar_ptr, norm_ptr, radial_ptr, n, fraction, score_ptr, stream) -> None:
    _check(library().tm_prescore(ctx, lib_id, polar_ptr, norm_ptr, radial_ptr, n, fraction, score_ptr, stream))


def tm_check(ctx, stream) -> None:
    _check(library().tm_check(ctx, stream))


def tm_autotune(ctx, params, frames_ptr, dtype, n, H, W, lib_ids, stream) -> int:
    ids = (ctypes.c_int32 * len(lib_ids))(*lib_ids)
    best = ctypes.c_int32()
    _check(library().tm_autotune(ctx, ctypes.byref(params), frames_ptr, dtype, n, H, W, ids, len(lib_ids),
                                 ctypes.byref(best), stream))
    return best.value


def tm_index_patterns(ctx, params, frames_ptr, dtype, n, H, W, centres_ptr, lib_ids, out_ptr, stream) -> dict:
    ids = (ctypes.c_int32 * len(lib_ids))(*lib_ids)
    st = tm_stats()
    _check(library().tm_index_patterns(ctx, ctypes.byref(params), frames_ptr, dtype, n, H, W, centres_ptr,
                                       ids, len(lib_ids), out_ptr, ctypes.byref(st), stream))
    return {name: getattr(st, name) for name, _ in tm_stats._fields_}


def tm_index_patterns_host(ctx, params, frames_ptr, dtype, n, H, W, centres_ptr, lib_ids, out_ptr,
                           chunk: int = 0) -> dict:
    ids = (ctypes.c_int32 * len(lib_ids))(*lib_ids)
    st = tm_stats()
    _check(library().tm_index_patterns_host(ctx, ctypes.byref(params), frames_ptr, dtype, n, H, W, centres_ptr,
                                            ids, len(lib_ids), out_ptr, chunk, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in tm_stats._fields_}


def tm_profile_enable(ctx, enable: bool) -> None:
    _check(library().tm_profile_enable(ctx, 1 if enable else 0))


def tm_profile_read(ctx, counters: bool = False):
    """Stage totals {stage: (ms, launches)}; with counters=True also the work counters
    ({"sparse_macs": multiply-adds the FP32 sparse kernel executed})."""
    p = tm_profile()
    _check(library().tm_profile_read(ctx, ctypes.byref(p)))
    stages = {STAGES[i]: (p.ms[i], p.launches[i]) for i in range(TM_STAGE_COUNT) if p.launches[i]}
    return (stages, {"sparse_macs": int(p.sparse_macs)}) if counters else stages


def tm_server_params_default() -> tm_server_params:
    p = tm_server_params()
    library().tm_server_params_default(ctypes.byref(p))
    return p


def tm_server_create(ctx, params: tm_server_params) -> int:
    h = _P()
    _check(library().tm_server_create(ctx, ctypes.byref(params), ctypes.byref(h)))
    return h.value


def tm_server_submit(server, req: tm_request) -> int:
    t = ctypes.c_uint64()
    _check(library().tm_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def tm_server_wait(server, ticket: int, timeout_ms: int = -1) -> dict:
    st = tm_request_status()
    _check(library().tm_server_wait(server, ticket, timeout_ms, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in tm_request_status._fields_}


def tm_server_cancel(server, ticket: int) -> None:
    _check(library().tm_server_cancel(server, ticket))


def tm_server_pause(server, paused: bool) -> None:
    _check(library().tm_server_pause(server, 1 if paused else 0))


def tm_server_destroy(server) -> None:
    library().tm_server_destroy(server)


class Server:
    """Serving loop over a Context: host frames in, host hits out (see tm_server_* in tmgb.h)."""

    def __init__(self, ctx: "Context", slots=3, tile_patterns=512, max_H=256, max_W=256, max_libs=2, max_top_n=5,
                 queue_bytes=0, blocking_submit=True, priority_slots=None, hbm_budget_bytes=0, reserve_sms=-1):
        p = tm_server_params_default()
        p.slots, p.tile_patterns, p.max_H, p.max_W = slots, tile_patterns, max_H, max_W
        p.max_libs, p.max_top_n, p.queue_bytes, p.blocking_submit = max_libs, max_top_n, queue_bytes, int(blocking_submit)
        p.priority_slots = (1 if slots > 1 else 0) if priority_slots is None else priority_slots
        p.hbm_budget_bytes, p.reserve_sms = hbm_budget_bytes, reserve_sms
        self.ctx = ctx
        self.handle = tm_server_create(ctx.handle, p)
        self._keep = {}

    def submit(self, frames, lib_ids, top_n=5, priority=0, out: np.ndarray | None = None, **kw) -> int:
        """frames: C-contiguous uint16/float32 [n][H][W] host array (pinned memory gives overlap),
        or a contiguous CUDA tensor on the context's device (frames already resident); returns
        the ticket.  The result array is returned by wait()."""
        if isinstance(lib_ids, int):
            lib_ids = [lib_ids]
        n, H, W = frames.shape
        if out is None:
            out = np.empty((len(lib_ids), n, top_n), dtype=HIT_DTYPE)
        ids = np.ascontiguousarray(lib_ids, dtype=np.int32)
        r = tm_request()
        if isinstance(frames, np.ndarray):
            r.frames_host = frames.ctypes.data
            r.dtype = TM_DTYPE_U16 if frames.dtype == np.uint16 else TM_DTYPE_F32
        else:
            if not frames.is_cuda or not frames.is_contiguous():
                raise ValueError("device frames must be a contiguous CUDA tensor")
            r.frames_dev = frames.data_ptr()
            r.dtype = _dtype_code(frames)
        r.H, r.W, r.n = H, W, n
        r.lib_ids = ids.ctypes.data
        r.n_libs = len(lib_ids)
        r.priority = priority
        r.params = make_params(top_n=top_n, **kw)
        r.out_host = out.ctypes.data
        t = tm_server_submit(self.handle, r)
        self._keep[t] = (frames, out, ids)
        return t

    def wait(self, ticket, timeout_ms=-1):
        st = tm_server_wait(self.handle, ticket, timeout_ms)
        frames, out, ids = self._keep.pop(ticket)
        return out, st

    def cancel(self, ticket):
        tm_server_cancel(self.handle, ticket)

    def pause(self, paused=True):
        tm_server_pause(self.handle, paused)

    def close(self):
        if self.handle:
            tm_server_destroy(self.handle)
            self.handle = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- torch-facing wrapper

def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dtype_code(t):
    import torch
    if t.dtype == torch.uint16:
        return TM_DTYPE_U16
    if t.dtype == torch.float32:
        return TM_DTYPE_F32
    raise TypeError("frames must be torch.uint16 or torch.float32")


def _host_buffer(a, what):
    """(address, dtype code or None) of a C-contiguous host numpy array or CPU torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what} must be C-contiguous")
        code = {np.dtype(np.uint16): TM_DTYPE_U16, np.dtype(np.float32): TM_DTYPE_F32}.get(a.dtype)
        return a.ctypes.data, code
    if a.device.type != "cpu" or not a.is_contiguous():
        raise ValueError(f"{what} must be a contiguous host tensor")
    import torch
    code = {torch.uint16: TM_DTYPE_U16, torch.float32: TM_DTYPE_F32}.get(a.dtype)
    return a.data_ptr(), code


def hits_to_numpy(hits) -> np.ndarray:
    """[..., N, 5] int32 tensor or array of tm_hit rows -> structured numpy array."""
    a = np.ascontiguousarray(hits) if isinstance(hits, np.ndarray) else hits.detach().cpu().contiguous().numpy()
    return a.view(HIT_DTYPE).reshape(a.shape[:-1])


class Context:
    """One tmgb context on a CUDA device (torch tensors in, torch tensors out)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.handle = tm_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle:
            tm_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile_enable(self, enable=True):
        tm_profile_enable(self.handle, enable)

    def profile_read(self, counters=False):
        return tm_profile_read(self.handle, counters)

    def load_library(self, ts, n_r, n_theta, dr=1.0, mirror=None, unit_intensity=False) -> int:
        return tm_load_library(self.handle, ts, n_r, n_theta, dr, mirror, unit_intensity)

    def unload_library(self, lib_id):
        tm_unload_library(self.handle, lib_id)

    def library_info(self, lib_id) -> dict:
        return tm_library_info_get(self.handle, lib_id)

    def library_export(self, lib_id) -> dict:
        return tm_library_export(self.handle, lib_id)

    def polar_transform(self, frames, n_r, n_theta, dr=1.0, gamma=0.5, subtract=0.0, cx=math.nan, cy=math.nan,
                        centres=None, stream=None, mask=None, threshold=0.0):
        """frames [n][H][W] -> (polar [n][n_r][n_theta], norm [n], radial [n][n_r]); centres: optional
        float32 [n][2] device tensor of per-pattern (cx, cy)."""
        import torch
        n, H, W = frames.shape
        dev = frames.device
        polar = torch.empty((n, n_r, n_theta), dtype=torch.float32, device=dev)
        norm = torch.empty((n,), dtype=torch.float32, device=dev)
        radial = torch.empty((n, n_r), dtype=torch.float32, device=dev)
        p = make_params(gamma, subtract, cx, cy, mask=mask, threshold=threshold)
        tm_polar_transform(self.handle, p, frames.data_ptr(), _dtype_code(frames), n, H, W,
                           None if centres is None else centres.data_ptr(), n_r, n_theta, dr,
                           polar.data_ptr(), norm.data_ptr(), radial.data_ptr(), _stream_ptr(stream))
        return polar, norm, radial

    def prefilter(self, lib_id, radial, fraction, stream=None):
        import torch
        K = self.library_info(lib_id)["n_templates"]
        n = radial.shape[0]
        words = (K + 31) // 32
        mask = torch.empty((n, words), dtype=torch.int32, device=radial.device)
        score = torch.empty((n, K), dtype=torch.float32, device=radial.device)
        tm_prefilter(self.handle, lib_id, radial.data_ptr(), n, fraction, mask.data_ptr(), score.data_ptr(),
                     _stream_ptr(stream))
        return mask, score

    def correlate(self, lib_id, polar, norm, mask=None, stream=None):
        import torch
        K = self.library_info(lib_id)["n_templates"]
        n = polar.shape[0]
        q = torch.empty((n, K), dtype=torch.float32, device=polar.device)
        s = torch.empty((n, K), dtype=torch.int32, device=polar.device)
        tm_correlate(self.handle, lib_id, polar.data_ptr(), norm.data_ptr(), n,
                     None if mask is None else mask.data_ptr(), q.data_ptr(), s.data_ptr(), _stream_ptr(stream))
        return q, s

    def prescore(self, lib_id, polar, norm, radial=None, fraction=1.0, stream=None):
        """BF16 tensor-core pre-score of every template: [n][K] float, NaN where not scored."""
        import torch
        n = polar.shape[0]
        K = self.library_info(lib_id)["n_templates"]
        score = torch.empty((n, K), dtype=torch.float32, device=polar.device)
        tm_prescore(self.handle, lib_id, polar.data_ptr(), norm.data_ptr(),
                    None if radial is None else radial.data_ptr(), n, fraction, score.data_ptr(), _stream_ptr(stream))
        return score

    def autotune(self, frames, lib_ids, top_n=5, prefilter=1.0, stream=None) -> int:
        """Pick the sparse kernel's block size for these libraries by timing; returns it."""
        if isinstance(lib_ids, int):
            lib_ids = [lib_ids]
        n, H, W = frames.shape
        p = make_params(top_n=top_n, prefilter=prefilter)
        return tm_autotune(self.handle, p, frames.data_ptr(), _dtype_code(frames), n, H, W, list(lib_ids),
                           _stream_ptr(stream))

    def find_centres(self, frames, radius=6.0, iterations=3, cx=math.nan, cy=math.nan, out=None, stream=None):
        """Direct-beam centre per pattern (device frames [n][H][W]) -> float32 [n][2] tensor."""
        import torch
        n, H, W = frames.shape
        if out is None:
            out = torch.empty((n, 2), dtype=torch.float32, device=frames.device)
        _check(library().tm_find_centres(self.handle, frames.data_ptr(), _dtype_code(frames), n, H, W, float(cx),
                                         float(cy), float(radius), int(iterations), out.data_ptr(),
                                         _stream_ptr(stream)))
        return out

    def orientation_vectors(self, hits, rot, K0, axis=(0.0, 0.0, 1.0), stream=None):
        """Crystal direction along the sample axis for each pattern's best hit: hits the
        [n][top_n][5] int32 device tensor of index(), rot [K0][3][3] float64 device tensor
        -> float64 [n][3] (NaN where no hit)."""
        import torch
        n, top_n = hits.shape[-3], hits.shape[-2]
        v = torch.empty((n, 3), dtype=torch.float64, device=hits.device)
        _check(library().tm_orientation_vectors(self.handle, hits.data_ptr(), n, top_n, rot.data_ptr(), int(K0),
                                                float(axis[0]), float(axis[1]), float(axis[2]), v.data_ptr(),
                                                _stream_ptr(stream)))
        return v

    def angular_deviation(self, va, vb, stream=None):
        """Eq. 2 per pattern in degrees (float64 device tensors [n][3] -> [n])."""
        import torch
        n = va.shape[0]
        d = torch.empty((n,), dtype=torch.float64, device=va.device)
        _check(library().tm_angular_deviation(self.handle, va.data_ptr(), vb.data_ptr(), n, d.data_ptr(),
                                              _stream_ptr(stream)))
        return d

    def kinematic_spots(self, g, f2, gnorm, rot, wavelength, s_max, max_spots, stream=None):
        """Reflections kept per orientation (device tensors: g [G][3], f2 [G], gnorm [G], rot
        [D][3][3], float64) -> (counts int32 [D], spots float64 [D][max_spots][3] = kx, ky, I)."""
        import torch
        D = rot.shape[0]
        counts = torch.empty((D,), dtype=torch.int32, device=rot.device)
        spots = torch.zeros((D, max_spots, 3), dtype=torch.float64, device=rot.device)
        _check(library().tm_kinematic_spots(self.handle, g.data_ptr(), f2.data_ptr(), gnorm.data_ptr(), g.shape[0],
                                            rot.data_ptr(), D, float(wavelength), float(s_max), int(max_spots),
                                            counts.data_ptr(), spots.data_ptr(), _stream_ptr(stream)))
        return counts, spots

    def kinematic_templates(self, g, f2, gnorm, rot, wavelength, s_max, max_spots=150, px_per_unit=100.0,
                            mirror=True):
        """The simulated templates (numpy inputs as for kinematic_spots) as a TemplateSet in
        (kx, ky) coordinates, ready for load_library."""
        import torch
        from . import synth
        dev = torch.device("cuda", torch.cuda.current_device())
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
        counts, spots = self.kinematic_spots(t(g), t(f2), t(gnorm), t(rot), wavelength, s_max, max_spots)
        counts, spots = counts.cpu().numpy(), spots.cpu().numpy()
        if np.any(counts < 0):
            raise TmError(TM_ERR_UNSUPPORTED, "more than %d reflections within s_max for an orientation" % 512)
        offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        flat = np.concatenate([spots[d, :counts[d]] for d in range(len(counts))]) if len(counts) else np.zeros((0, 3))
        return synth.TemplateSet(offsets, flat[:, 0].copy(), flat[:, 1].copy(), flat[:, 2].copy(), coords="xy",
                                 px_per_unit=px_per_unit, mirror=mirror, meta={"kind": "kinematic (device)"})

    def preprocess(self, frames, dog=None, blur=0.0, truncate=4.0, out=None, stream=None):
        """Background removal (difference of Gaussians, dog = (sigma_min, sigma_max)) and
        Gaussian blur of device frames [n][H][W] -> float32 [n][H][W] tensor."""
        import torch
        n, H, W = frames.shape
        if out is None:
            out = torch.empty((n, H, W), dtype=torch.float32, device=frames.device)
        p = tm_preprocess_params(float(dog[0]) if dog else 0.0, float(dog[1]) if dog else 0.0, float(blur),
                                 float(truncate))
        _check(library().tm_preprocess(self.handle, ctypes.byref(p), frames.data_ptr(), _dtype_code(frames), n, H, W,
                                       out.data_ptr(), _stream_ptr(stream)))
        return out

    def frame_sum(self, frames, out=None, accumulate=False, stream=None):
        """Per-pixel FP64 sum over frames [n][H][W] (device) -> [H][W] float64 tensor; with
        accumulate=True the sums are added onto `out`."""
        import torch
        n, H, W = frames.shape
        if out is None:
            out = torch.zeros((H, W), dtype=torch.float64, device=frames.device)
        _check(library().tm_frame_sum(self.handle, frames.data_ptr(), _dtype_code(frames), n, H, W,
                                      1 if accumulate else 0, out.data_ptr(), _stream_ptr(stream)))
        return out

    def matrix_mask(self, sums, n_frames, threshold, n_open=1, n_dilate=2, stream=None):
        """Mask of kept pixels (uint8 [H][W] device tensor, 1 = keep) from per-pixel sums."""
        import torch
        H, W = sums.shape
        mask = torch.empty((H, W), dtype=torch.uint8, device=sums.device)
        _check(library().tm_matrix_mask(self.handle, sums.data_ptr(), n_frames, H, W, float(threshold), n_open,
                                        n_dilate, mask.data_ptr(), _stream_ptr(stream)))
        return mask

    def check(self, stream=None):
        """Synchronise and raise TmError(TM_ERR_TIMEOUT) if a kernel stopped on a bounded wait."""
        tm_check(self.handle, _stream_ptr(stream))

    def index_host(self, frames, lib_ids, top_n=5, gamma=0.5, subtract=0.0, prefilter=1.0,
                   path=TM_PATH_FP32_SPARSE, rescore_k=256, cx=math.nan, cy=math.nan, out=None, chunk=0,
                   centres=None, mask=None, threshold=0.0):
        """frames [n][H][W] uint16/float32 in host memory (numpy, or a CPU tensor -- pinned for
        copy/compute overlap) -> hits [n_libs][n][top_n][5] int32 in host memory (`out`, numpy
        or CPU tensor, else a new numpy array).  Synchronous."""
        if isinstance(lib_ids, int):
            lib_ids = [lib_ids]
        n, H, W = frames.shape
        fptr, code = _host_buffer(frames, "frames")
        if code is None:
            raise TypeError("frames must be uint16 or float32")
        if out is None:
            out = np.empty((len(lib_ids), n, top_n, 5), dtype=np.int32)
        if tuple(out.shape) != (len(lib_ids), n, top_n, 5):
            raise ValueError("out must have shape [n_libs][n][top_n][5]")
        optr, _ = _host_buffer(out, "out")
        cptr = None
        if centres is not None:
            cptr, ccode = _host_buffer(centres, "centres")
            if ccode != TM_DTYPE_F32 or tuple(centres.shape) != (n, 2):
                raise ValueError("centres must be float32 [n][2]")
        p = make_params(gamma, subtract, cx, cy, prefilter, top_n, path, rescore_k, mask=mask, threshold=threshold)
        self.last_stats = tm_index_patterns_host(self.handle, p, fptr, code, n, H, W, cptr, list(lib_ids), optr,
                                                 chunk)
        return out

    def index(self, frames, lib_ids, top_n=5, gamma=0.5, subtract=0.0, prefilter=1.0,
              path=TM_PATH_FP32_SPARSE, rescore_k=256, cx=math.nan, cy=math.nan, out=None, stream=None,
              graph=False, centres=None, test_stall=False, mask=None, threshold=0.0, refine=False):
        """frames [n][H][W] uint16/float32 on the device -> hits [n_libs][n][top_n][5] int32.
        graph=True replays repeated identical calls as a CUDA graph (needs a created stream).
        test_stall=True sets TM_INDEX_TEST_STALL (failure-path tests of the bounded waits)."""
        import torch
        if isinstance(lib_ids, int):
            lib_ids = [lib_ids]
        n, H, W = frames.shape
        if out is None:
            out = torch.empty((len(lib_ids), n, top_n, 5), dtype=torch.int32, device=frames.device)
        p = make_params(gamma, subtract, cx, cy, prefilter, top_n, path, rescore_k, mask=mask, threshold=threshold)
        if graph:
            p.reserved |= TM_INDEX_GRAPH
        if test_stall:
            p.reserved |= TM_INDEX_TEST_STALL
        if refine:
            p.reserved |= TM_INDEX_REFINE
        self.last_stats = tm_index_patterns(self.handle, p, frames.data_ptr(), _dtype_code(frames), n, H, W,
                                            None if centres is None else centres.data_ptr(),
                                            list(lib_ids), out.data_ptr(), _stream_ptr(stream))
        return out
