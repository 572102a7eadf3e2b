"""ctypes binding of libtdpm (include/tdpm.h): the same entry points, argument marshalling only.

Every step of the scoring path runs in the library's CUDA kernels; this module only converts Python objects (numpy
host arrays, torch CUDA tensors, streams) into the C structs and pointers, and turns non-zero status codes into
``TdpmError``. Importing it loads ``_build/libtdpm.so`` and fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

FEAT_DIM = 32
MAX_PARTS = 16

OK, ERR_ARG, ERR_SHAPE, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT, ERR_CUDA, ERR_STATE, ERR_IO = 0, -1, -2, -3, -4, -5, -6, -7, -8
FORM_FULL, FORM_DECOMPOSED = 0, 1
PREC_FP32, PREC_BF16, PREC_FP8, PREC_BF16X3 = 0, 1, 2, 3
DECOMP_PER_FILTER, DECOMP_JOINT = 0, 1
MAP_FILTER_SCORE, MAP_FINAL_SCORE, MAP_PART_DT, MAP_PART_ARG = 0, 1, 2, 3

_c_i32 = ctypes.c_int32
_c_f32p = ctypes.POINTER(ctypes.c_float)


class TdpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tdpm status {status}: {msg}")
        self.status = status


class Filter(ctypes.Structure):
    _fields_ = [("h", _c_i32), ("w", _c_i32), ("data", _c_f32p)]


class Part(ctypes.Structure):
    _fields_ = [("filter", Filter), ("anchor_y", _c_i32), ("anchor_x", _c_i32), ("deform", ctypes.c_float * 4)]


class Component(ctypes.Structure):
    _fields_ = [("root", Filter), ("bias", ctypes.c_float), ("n_parts", _c_i32), ("parts", ctypes.POINTER(Part))]


class ModelDesc(ctypes.Structure):
    _fields_ = [("n_components", _c_i32), ("components", ctypes.POINTER(Component))]


class Level(ctypes.Structure):
    _fields_ = [("H", _c_i32), ("W", _c_i32), ("data", ctypes.c_void_p)]


class PyramidDesc(ctypes.Structure):
    _fields_ = [("n_levels", _c_i32), ("lambda_", _c_i32), ("levels", ctypes.POINTER(Level))]


class Detection(ctypes.Structure):
    _fields_ = [("image", _c_i32), ("model", _c_i32), ("component", _c_i32), ("level", _c_i32), ("y", _c_i32),
                ("x", _c_i32), ("score", ctypes.c_float), ("n_parts", _c_i32), ("part_y", _c_i32 * MAX_PARTS),
                ("part_x", _c_i32 * MAX_PARTS)]


class Request(ctypes.Structure):
    _fields_ = [("pyramid", ctypes.POINTER(PyramidDesc)), ("model_ids", ctypes.POINTER(_c_i32)), ("n_models", _c_i32),
                ("form", _c_i32), ("precision", _c_i32), ("tau", ctypes.c_float),
                ("components", ctypes.POINTER(_c_i32)), ("n_components", _c_i32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch_images", _c_i32), ("max_inflight", _c_i32), ("max_wait_us", _c_i32),
                ("mem_budget_bytes", ctypes.c_size_t)]


class ResultInfo(ctypes.Structure):
    _fields_ = [("status", _c_i32), ("batch_images", _c_i32), ("t_submit_ns", ctypes.c_uint64),
                ("t_start_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64), ("n_detections", ctypes.c_uint64)]


class DecompReport(ctypes.Structure):
    _fields_ = [("n_groups", _c_i32), ("total_rank", _c_i32), ("total_iters", _c_i32),
                ("max_rel_error", ctypes.c_double), ("mean_rel_error", ctypes.c_double), ("gain", ctypes.c_double)]


class CascadeStats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("pruned", ctypes.c_int64), ("terms_evaluated", ctypes.c_int64),
                ("terms_total", ctypes.c_int64)]


DETECTION_DTYPE = np.dtype([("image", np.int32), ("model", np.int32), ("component", np.int32), ("level", np.int32),
                            ("y", np.int32), ("x", np.int32), ("score", np.float32), ("n_parts", np.int32),
                            ("part_y", np.int32, MAX_PARTS), ("part_x", np.int32, MAX_PARTS)])
assert DETECTION_DTYPE.itemsize == ctypes.sizeof(Detection)

# every symbol include/tdpm.h declares, with (restype, argtypes)
_VP = ctypes.c_void_p
SIGNATURES = {
    "tdpm_create": (_c_i32, [ctypes.POINTER(_VP), _c_i32, ctypes.c_size_t]),
    "tdpm_destroy": (None, [_VP]),
    "tdpm_last_error": (ctypes.c_char_p, []),
    "tdpm_version": (ctypes.c_char_p, []),
    "tdpm_load_model": (_c_i32, [_VP, ctypes.POINTER(ModelDesc), ctypes.POINTER(_c_i32)]),
    "tdpm_model_info": (_c_i32, [_VP, _c_i32, ctypes.POINTER(_c_i32), ctypes.POINTER(_c_i32)]),
    "tdpm_group_info": (_c_i32, [_VP, _c_i32, _c_i32] + [ctypes.POINTER(_c_i32)] * 6 + [_c_i32]),
    "tdpm_decompose": (_c_i32, [_VP, _c_i32, _c_i32, _c_i32, _c_i32, ctypes.c_double, ctypes.c_uint64,
                                ctypes.POINTER(DecompReport)]),
    "tdpm_decompose_auto": (_c_i32, [_VP, _c_i32, ctypes.c_double, _c_i32, _c_i32, ctypes.c_double, ctypes.c_uint64,
                                     _VP, ctypes.POINTER(DecompReport)]),
    "tdpm_decompose_ranks": (_c_i32, [_VP, _c_i32, _VP, _c_i32, ctypes.c_double, ctypes.c_uint64,
                                      ctypes.POINTER(DecompReport)]),
    "tdpm_get_factors": (_c_i32, [_VP, _c_i32, _c_i32] + [ctypes.POINTER(ctypes.c_double)] * 4),
    "tdpm_save_factors": (_c_i32, [_VP, _c_i32, ctypes.c_char_p]),
    "tdpm_load_factors": (_c_i32, [_VP, _c_i32, ctypes.c_char_p]),
    "tdpm_build_pyramid_scores": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _c_i32, _VP,
                                           ctypes.POINTER(_c_i32)]),
    "tdpm_detect": (_c_i32, [_VP, _c_i32, ctypes.c_float, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _VP]),
    "tdpm_detect_thresholds": (_c_i32, [_VP, _c_i32, _VP, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                        _VP]),
    "tdpm_build_batch_scores": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _c_i32, _c_i32, _VP,
                                         ctypes.POINTER(_c_i32)]),
    "tdpm_build_batch_scores_subset": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _VP, _c_i32, _c_i32,
                                                _VP, ctypes.POINTER(_c_i32)]),
    "tdpm_scores_bytes": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _c_i32, _c_i32,
                                   ctypes.POINTER(ctypes.c_size_t)]),
    "tdpm_server_start": (_c_i32, [_VP, ctypes.POINTER(ServerConfig)]),
    "tdpm_server_stop": (_c_i32, [_VP]),
    "tdpm_submit": (_c_i32, [_VP, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "tdpm_poll": (_c_i32, [_VP, ctypes.c_uint64, _c_i32, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                           ctypes.POINTER(ResultInfo)]),
    "tdpm_get_maps": (_c_i32, [_VP, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _VP, ctypes.c_size_t,
                               ctypes.POINTER(_c_i32), ctypes.POINTER(_c_i32), _VP]),
    "tdpm_release": (_c_i32, [_VP, _c_i32]),
    "tdpm_dt_scratch_bytes": (ctypes.c_size_t, [_c_i32, _c_i32]),
    "tdpm_dt": (_c_i32, [_VP, _c_i32, _c_i32, _c_f32p, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _VP, _VP, _VP,
                         _VP]),
    "tdpm_correlate": (_c_i32, [_VP, _c_i32, _c_i32, _c_f32p, _c_i32, _c_i32, _c_i32, _c_i32, _VP, _VP]),
    "tdpm_dt_noalloc_max_elements": (ctypes.c_size_t, []),
    "tdpm_dt_noalloc": (_c_i32, [_VP, _c_i32, _c_i32, _c_f32p, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _VP,
                                 _VP, _VP]),
    "tdpm_kernel_launches": (ctypes.c_uint64, []),
    "tdpm_profile_enable": (_c_i32, [_VP, _c_i32]),
    "tdpm_set_fusion": (_c_i32, [_VP, _c_i32]),
    "tdpm_selftest_bounded_wait": (_c_i32, [_VP]),
    "tdpm_detect_nms": (_c_i32, [_VP, _c_i32, ctypes.c_float, _VP, ctypes.c_double, ctypes.c_double, _VP,
                                 ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _VP]),
    "tdpm_cascade_partials": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _VP, ctypes.c_size_t, _VP,
                                       _c_i32, _c_i32, _VP]),
    "tdpm_cascade_thresholds": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _VP, ctypes.c_size_t, _VP,
                                         _c_i32, _VP]),
    "tdpm_detect_cascade": (_c_i32, [_VP, _c_i32, ctypes.POINTER(PyramidDesc), _c_i32, _VP, _c_i32, ctypes.c_float,
                                     _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(CascadeStats), _VP]),
    "tdpm_hog_pyramid_shape": (_c_i32, [_c_i32, _c_i32, _c_i32, _c_i32, _c_i32, ctypes.POINTER(_c_i32), _VP, _c_i32,
                                        ctypes.POINTER(ctypes.c_size_t)]),
    "tdpm_hog_pyramid": (_c_i32, [_VP, _VP, _c_i32, _c_i32, _c_i32, _c_i32, _c_i32, _VP, ctypes.c_size_t,
                                  ctypes.POINTER(Level), _c_i32, ctypes.POINTER(_c_i32), _VP]),
    "tdpm_hog_features": (_c_i32, [_VP, _VP, _c_i32, _c_i32, _c_i32, _VP, ctypes.c_size_t, ctypes.POINTER(_c_i32),
                                   ctypes.POINTER(_c_i32), _VP]),
    "tdpm_resize": (_c_i32, [_VP, _VP, _c_i32, _c_i32, ctypes.c_double, _VP, ctypes.c_size_t, ctypes.POINTER(_c_i32),
                             ctypes.POINTER(_c_i32), _VP]),
    "tdpm_profile_read": (_c_i32, [_VP, _c_i32, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_c_i32)]),
    "tdpm_profile_reset": (_c_i32, [_VP]),
    "tdpm_autotune_read": (_c_i32, [_VP, _c_i32, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(_c_i32),
                                    ctypes.POINTER(_c_i32), ctypes.POINTER(_c_i32)]),
}

_LIB: Optional[ctypes.CDLL] = None


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libtdpm.so (built by ``paper_1707_03268_gb300.build``); raise if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libtdpm.so is not built ({_build.LIB}); run __graft_entry__.build() first")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(st: int) -> None:
    if st != OK:
        raise TdpmError(st, lib().tdpm_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    """Device pointer of a torch tensor (or an int)."""
    return t if isinstance(t, int) else int(t.data_ptr())


# --------------------------------------------------------------------------------------------------- context
def tdpm_create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().tdpm_create(ctypes.byref(h), int(device), int(mem_budget_bytes)))
    return h.value


def tdpm_destroy(ctx: int) -> None:
    lib().tdpm_destroy(ctx)


def tdpm_last_error() -> str:
    return lib().tdpm_last_error().decode(errors="replace")


def tdpm_version() -> str:
    return lib().tdpm_version().decode()


# --------------------------------------------------------------------------------------------------- model
def _filter(arr: np.ndarray, keep: list) -> Filter:
    a = np.ascontiguousarray(arr, dtype=np.float32)
    assert a.ndim == 3 and a.shape[2] == FEAT_DIM
    keep.append(a)
    return Filter(a.shape[0], a.shape[1], a.ctypes.data_as(_c_f32p))


def tdpm_load_model(ctx: int, model) -> int:
    """Load a model given as an object with ``components`` (each with ``root``, ``parts`` [filt, anchor, deform],
    ``bias``), e.g. ``synth.Model``."""
    keep: list = []
    comps = (Component * len(model.components))()
    for i, c in enumerate(model.components):
        parts = (Part * max(1, len(c.parts)))()
        for k, p in enumerate(c.parts):
            parts[k] = Part(_filter(p.filt, keep), int(p.anchor[0]), int(p.anchor[1]),
                            (ctypes.c_float * 4)(*[float(v) for v in p.deform]))
        keep.append(parts)
        comps[i] = Component(_filter(c.root, keep), float(c.bias), len(c.parts), parts)
    desc = ModelDesc(len(model.components), comps)
    mid = _c_i32()
    _check(lib().tdpm_load_model(ctx, ctypes.byref(desc), ctypes.byref(mid)))
    return mid.value


def tdpm_model_info(ctx: int, model_id: int) -> Tuple[int, int]:
    nf, ng = _c_i32(), _c_i32()
    _check(lib().tdpm_model_info(ctx, model_id, ctypes.byref(nf), ctypes.byref(ng)))
    return nf.value, ng.value


def tdpm_group_info(ctx: int, model_id: int, group: int) -> dict:
    role, h, w, n, rank = (_c_i32() for _ in range(5))
    _check(lib().tdpm_group_info(ctx, model_id, group, ctypes.byref(role), ctypes.byref(h), ctypes.byref(w),
                                 ctypes.byref(n), ctypes.byref(rank), None, 0))
    ids = (_c_i32 * n.value)()
    _check(lib().tdpm_group_info(ctx, model_id, group, None, None, None, None, None, ids, n.value))
    return {"role": role.value, "h": h.value, "w": w.value, "n_filters": n.value, "rank": rank.value,
            "filter_ids": list(ids)}


def tdpm_decompose(ctx: int, model_id: int, rank: int, mode: int = DECOMP_PER_FILTER, max_iters: int = 500,
                   tol: float = 1e-10, seed: int = 0) -> dict:
    rep = DecompReport()
    _check(lib().tdpm_decompose(ctx, model_id, int(rank), int(mode), int(max_iters), float(tol), int(seed),
                                ctypes.byref(rep)))
    return {f: getattr(rep, f) for f, _ in DecompReport._fields_}


def tdpm_decompose_ranks(ctx: int, model_id: int, ranks, max_iters: int = 500, tol: float = 1e-10,
                         seed: int = 0) -> dict:
    """Per-filter decomposition with one rank per filter (by filter id), e.g. Sec. 5's (S, T) root / part ranks."""
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.int32))
    rep = DecompReport()
    _check(lib().tdpm_decompose_ranks(ctx, model_id, r.ctypes.data, int(max_iters), float(tol), int(seed),
                                      ctypes.byref(rep)))
    return {f: getattr(rep, f) for f, _ in DecompReport._fields_}


def tdpm_decompose_auto(ctx: int, model_id: int, e: float, max_rank: int, max_iters: int = 500, tol: float = 1e-10,
                        seed: int = 0) -> Tuple[dict, np.ndarray]:
    """Per-filter decomposition at the smallest rank meeting the paper's rank criterion with constant e (Sec. 4).
    Returns the report and the chosen rank of every filter (by filter id)."""
    n_f, _ = tdpm_model_info(ctx, model_id)
    ranks = np.zeros(n_f, dtype=np.int32)
    rep = DecompReport()
    _check(lib().tdpm_decompose_auto(ctx, model_id, float(e), int(max_rank), int(max_iters), float(tol), int(seed),
                                     ranks.ctypes.data, ctypes.byref(rep)))
    return {f: getattr(rep, f) for f, _ in DecompReport._fields_}, ranks


def tdpm_get_factors(ctx: int, model_id: int, group: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    info = tdpm_group_info(ctx, model_id, group)
    R, h, w, K = info["rank"], info["h"], info["w"], info["n_filters"]
    A, B, C, Lam = (np.zeros((n, R)) for n in (h, w, FEAT_DIM, K))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().tdpm_get_factors(ctx, model_id, group, A.ctypes.data_as(dp), B.ctypes.data_as(dp),
                                  C.ctypes.data_as(dp), Lam.ctypes.data_as(dp)))
    return A, B, C, Lam


def tdpm_save_factors(ctx: int, model_id: int, path: str) -> None:
    _check(lib().tdpm_save_factors(ctx, model_id, path.encode()))


def tdpm_load_factors(ctx: int, model_id: int, path: str) -> None:
    _check(lib().tdpm_load_factors(ctx, model_id, path.encode()))


# --------------------------------------------------------------------------------------------------- scoring
class DevicePyramid:
    """Levels of a feature pyramid as torch CUDA tensors ([H][W][32] FP32, contiguous) plus lambda."""

    def __init__(self, levels: Sequence, lam: int):
        self.levels = list(levels)
        self.lam = int(lam)
        arr = (Level * len(self.levels))()
        for i, t in enumerate(self.levels):
            assert t.dim() == 3 and t.shape[2] == FEAT_DIM and t.is_contiguous() and t.is_cuda
            arr[i] = Level(int(t.shape[0]), int(t.shape[1]), _ptr(t))
        self._arr = arr
        self.desc = PyramidDesc(len(self.levels), self.lam, arr)


def tdpm_build_pyramid_scores(ctx: int, model_id: int, pyramid: DevicePyramid, form: int = FORM_FULL,
                              precision: int = PREC_FP32, stream=None) -> int:
    sid = _c_i32()
    _check(lib().tdpm_build_pyramid_scores(ctx, model_id, ctypes.byref(pyramid.desc), int(form), int(precision),
                                           _stream_ptr(stream), ctypes.byref(sid)))
    return sid.value


def tdpm_build_batch_scores(ctx: int, model_id: int, pyramids: Sequence[DevicePyramid], form: int = FORM_FULL,
                            precision: int = PREC_FP32, stream=None) -> int:
    """Score a batch of pyramids in one scores set (detections carry the image index)."""
    arr = (PyramidDesc * len(pyramids))(*[p.desc for p in pyramids])
    sid = _c_i32()
    _check(lib().tdpm_build_batch_scores(ctx, model_id, arr, len(pyramids), int(form), int(precision),
                                         _stream_ptr(stream), ctypes.byref(sid)))
    return sid.value


def tdpm_detect(ctx: int, scores_id: int, tau: float, capacity: int = 1 << 20, stream=None,
                out: Optional[np.ndarray] = None) -> np.ndarray:
    """Detections with score >= tau as a structured array (DETECTION_DTYPE), ordered by (component, level, y, x).
    Raises TdpmError(ERR_CAPACITY) when more than ``capacity`` exist."""
    if out is None or out.shape[0] < capacity:
        out = np.zeros(capacity, dtype=DETECTION_DTYPE)
    n = ctypes.c_size_t()
    st = lib().tdpm_detect(ctx, scores_id, float(tau), out.ctypes.data if capacity else None, int(capacity),
                           ctypes.byref(n), _stream_ptr(stream))
    _check(st)
    return out[: n.value]


def tdpm_detect_nms(ctx: int, scores_id: int, tau: float, component_class: Optional[Sequence[int]] = None,
                    overlap: float = 0.5, cell0: float = 4.0, capacity: int = 1 << 20, stream=None,
                    out: Optional[np.ndarray] = None) -> np.ndarray:
    """Detections with score >= tau after greedy non-maximum suppression per (image, class) on the device."""
    if out is None or out.shape[0] < capacity:
        out = np.zeros(capacity, dtype=DETECTION_DTYPE)
    cls = None if component_class is None else np.ascontiguousarray(component_class, dtype=np.int32)
    n = ctypes.c_size_t()
    _check(lib().tdpm_detect_nms(ctx, scores_id, float(tau), None if cls is None else cls.ctypes.data, float(overlap),
                                 float(cell0), out.ctypes.data if capacity else None, int(capacity), ctypes.byref(n),
                                 _stream_ptr(stream)))
    return out[: n.value]


def _pyr_array(pyramids: Sequence[DevicePyramid]):
    return (PyramidDesc * len(pyramids))(*[p.desc for p in pyramids])


def cascade_terms_bound(ctx: int, model_id: int) -> int:
    """An upper bound on any filter's number of CP terms: per shape group min(the group's terms, h * w)."""
    _, ng = tdpm_model_info(ctx, model_id)
    return max(min(g["rank"], g["h"] * g["w"]) for g in (tdpm_group_info(ctx, model_id, i) for i in range(ng)))


def _records(recs: np.ndarray) -> np.ndarray:
    recs = np.ascontiguousarray(recs)
    assert recs.dtype == DETECTION_DTYPE
    return recs


def tdpm_cascade_partials(ctx: int, scores_id: int, pyramids: Sequence[DevicePyramid], records: np.ndarray,
                          model_id: int, stream=None) -> np.ndarray:
    """Partial sums [n][1 + MAX_PARTS][T] of every filter of each record's component (slot 0 root, 1 + p part p), T =
    cascade_terms_bound; NaN where a filter has fewer terms or slots."""
    recs = _records(records)
    T = cascade_terms_bound(ctx, model_id)
    out = np.empty((max(len(recs), 1), 1 + MAX_PARTS, T), np.float32)
    _check(lib().tdpm_cascade_partials(ctx, scores_id, _pyr_array(pyramids), len(pyramids), recs.ctypes.data,
                                       len(recs), out.ctypes.data, 1 + MAX_PARTS, T, _stream_ptr(stream)))
    return out[: len(recs)]


def tdpm_cascade_thresholds(ctx: int, scores_id: int, pyramids: Sequence[DevicePyramid], positives: np.ndarray,
                            model_id: int, stream=None) -> np.ndarray:
    """Sec. 4 thresholds [n_filters][T] from positive records (-inf for filters without positives and beyond a
    filter's rank)."""
    recs = _records(positives)
    T = cascade_terms_bound(ctx, model_id)
    nf, _ = tdpm_model_info(ctx, model_id)
    t = np.empty((nf, T), np.float32)
    _check(lib().tdpm_cascade_thresholds(ctx, scores_id, _pyr_array(pyramids), len(pyramids), recs.ctypes.data,
                                         len(recs), t.ctypes.data, T, _stream_ptr(stream)))
    return t


def tdpm_detect_cascade(ctx: int, scores_id: int, pyramids: Sequence[DevicePyramid], thresholds: np.ndarray,
                        tau: float, capacity: int = 1 << 20, stream=None,
                        out: Optional[np.ndarray] = None) -> Tuple[np.ndarray, dict]:
    """Detections with score >= tau that the convolution-shortening cascade keeps, and its pruning counts."""
    t = np.ascontiguousarray(thresholds, dtype=np.float32)
    if out is None or out.shape[0] < capacity:
        out = np.zeros(capacity, dtype=DETECTION_DTYPE)
    n = ctypes.c_size_t()
    st = CascadeStats()
    _check(lib().tdpm_detect_cascade(ctx, scores_id, _pyr_array(pyramids), len(pyramids), t.ctypes.data,
                                     int(t.shape[1]), float(tau), out.ctypes.data if capacity else None,
                                     int(capacity), ctypes.byref(n), ctypes.byref(st), _stream_ptr(stream)))
    return out[: n.value], {f: getattr(st, f) for f, _ in CascadeStats._fields_}


def tdpm_hog_pyramid_shape(img_h: int, img_w: int, sbin: int = 8, lam: int = 10,
                           min_cells: int = 8) -> Tuple[List[Tuple[int, int]], int]:
    """Level sizes (rows, columns) and output bytes of the HOG pyramid of an img_h x img_w image."""
    n = _c_i32()
    b = ctypes.c_size_t()
    _check(lib().tdpm_hog_pyramid_shape(img_h, img_w, sbin, lam, min_cells, ctypes.byref(n), None, 0, ctypes.byref(b)))
    hw = (_c_i32 * (2 * n.value))()
    _check(lib().tdpm_hog_pyramid_shape(img_h, img_w, sbin, lam, min_cells, ctypes.byref(n), hw, n.value,
                                        ctypes.byref(b)))
    return [(hw[2 * j], hw[2 * j + 1]) for j in range(n.value)], b.value


class HogPyramid(DevicePyramid):
    """The device feature pyramid of an img_h x img_w image: level views of one flat FP32 CUDA tensor, filled by
    ``compute`` (one library call; repeated calls with the same image buffer replay the library's cached launches)."""

    def __init__(self, img_h: int, img_w: int, sbin: int = 8, lam: int = 10, min_cells: int = 8, out=None,
                 device="cuda"):
        import torch
        shapes, nbytes = tdpm_hog_pyramid_shape(img_h, img_w, sbin, lam, min_cells)
        if out is None:
            out = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
        assert out.is_cuda and out.dtype == torch.float32 and out.numel() * 4 >= nbytes and out.is_contiguous()
        levels, off = [], 0
        for (h, w) in shapes:
            levels.append(out[off:off + h * w * FEAT_DIM].view(h, w, FEAT_DIM))
            off += h * w * FEAT_DIM
        super().__init__(levels, lam)
        self.flat, self.nbytes = out, nbytes
        self.img_hw, self.sbin, self.min_cells = (img_h, img_w), sbin, min_cells
        self._hog_levels = (Level * len(shapes))()
        self._n = _c_i32()

    def compute(self, ctx: int, image, stream=None) -> "HogPyramid":
        """Fill the levels from a CUDA uint8 image [img_h][img_w][3] (contiguous)."""
        assert tuple(image.shape) == (self.img_hw[0], self.img_hw[1], 3) and image.is_contiguous()
        _check(lib().tdpm_hog_pyramid(ctx, image.data_ptr(), self.img_hw[0], self.img_hw[1], self.sbin, self.lam,
                                      self.min_cells, self.flat.data_ptr(), self.nbytes, self._hog_levels,
                                      len(self.levels), ctypes.byref(self._n), _stream_ptr(stream)))
        return self


def tdpm_hog_pyramid(ctx: int, image, sbin: int = 8, lam: int = 10, min_cells: int = 8, out=None,
                     stream=None, pyramid: Optional["HogPyramid"] = None) -> "HogPyramid":
    """HOG feature pyramid of a CUDA uint8 tensor [H][W][3] as a DevicePyramid ready for scoring (``pyramid``: one
    made before for the same image size, reused)."""
    import torch
    assert image.is_cuda and image.dtype == torch.uint8 and image.dim() == 3 and image.shape[2] == 3
    image = image.contiguous()
    if pyramid is None:
        pyramid = HogPyramid(int(image.shape[0]), int(image.shape[1]), sbin, lam, min_cells, out, image.device)
    return pyramid.compute(ctx, image, stream)


def tdpm_hog_features(ctx: int, img, sbin: int, stream=None):
    """32-channel features of one CUDA FP32 image [h][w][3] at cell size sbin (a CUDA tensor [h'][w'][32])."""
    import torch
    assert img.is_cuda and img.dtype == torch.float32 and img.dim() == 3 and img.shape[2] == 3
    img = img.contiguous()
    h, w = int(img.shape[0]), int(img.shape[1])
    cy, cx = (2 * h + sbin) // (2 * sbin), (2 * w + sbin) // (2 * sbin)
    out = torch.empty((max(cy - 2, 0), max(cx - 2, 0), FEAT_DIM), dtype=torch.float32, device=img.device)
    oh, ow = _c_i32(), _c_i32()
    _check(lib().tdpm_hog_features(ctx, _ptr(img), h, w, sbin, _ptr(out) if out.numel() else _ptr(img),
                                   out.numel() * 4, ctypes.byref(oh), ctypes.byref(ow), _stream_ptr(stream)))
    return out


def tdpm_resize(ctx: int, img, scale: float, stream=None):
    """Area-averaging resample of a CUDA FP32 image [h][w][3] by scale in (0, 1]."""
    import math as _m
    import torch
    assert img.is_cuda and img.dtype == torch.float32 and img.dim() == 3 and img.shape[2] == 3
    img = img.contiguous()
    h, w = int(img.shape[0]), int(img.shape[1])
    ho, wo = int(_m.floor(h * scale + 0.5)), int(_m.floor(w * scale + 0.5))
    out = torch.empty((max(ho, 1), max(wo, 1), 3), dtype=torch.float32, device=img.device)
    oh, ow = _c_i32(), _c_i32()
    _check(lib().tdpm_resize(ctx, _ptr(img), h, w, float(scale), _ptr(out), out.numel() * 4, ctypes.byref(oh),
                             ctypes.byref(ow), _stream_ptr(stream)))
    return out[: oh.value, : ow.value]


def tdpm_build_batch_scores_subset(ctx: int, model_id: int, pyramids: Sequence[DevicePyramid],
                                   component_mask: np.ndarray, form: int = FORM_FULL, precision: int = PREC_FP32,
                                   stream=None) -> int:
    """tdpm_build_batch_scores for the components marked in component_mask ([images][components], nonzero = yes)."""
    arr = (PyramidDesc * len(pyramids))(*[p.desc for p in pyramids])
    mask = np.ascontiguousarray(component_mask, dtype=np.uint8)
    sid = _c_i32()
    _check(lib().tdpm_build_batch_scores_subset(ctx, model_id, arr, len(pyramids), mask.ctypes.data, int(form),
                                                int(precision), _stream_ptr(stream), ctypes.byref(sid)))
    return sid.value


def tdpm_scores_bytes(ctx: int, model_id: int, pyramids: Sequence[DevicePyramid], form: int = FORM_FULL,
                      precision: int = PREC_FP32) -> int:
    """Device bytes a batch of these pyramids would hold (nothing is launched)."""
    arr = (PyramidDesc * len(pyramids))(*[p.desc for p in pyramids])
    b = ctypes.c_size_t()
    _check(lib().tdpm_scores_bytes(ctx, model_id, arr, len(pyramids), int(form), int(precision), ctypes.byref(b)))
    return b.value


# --------------------------------------------------------------------------------------------------- serving
_inflight_requests: Dict[Tuple[int, int], object] = {}  # (ctx, ticket) -> device pyramid kept alive until polled


def tdpm_server_start(ctx: int, max_batch_images: int = 16, max_inflight: int = 2, max_wait_us: int = 200,
                      mem_budget_bytes: int = 0) -> None:
    cfg = ServerConfig(int(max_batch_images), int(max_inflight), int(max_wait_us), int(mem_budget_bytes))
    _check(lib().tdpm_server_start(ctx, ctypes.byref(cfg)))


def tdpm_server_stop(ctx: int) -> None:
    _check(lib().tdpm_server_stop(ctx))


def tdpm_submit(ctx: int, pyramid: DevicePyramid, model_ids: Sequence[int], form: int = FORM_FULL,
                precision: int = PREC_FP32, tau: float = 0.0, components: Optional[Sequence[int]] = None) -> int:
    """Queue one request (an image pyramid on the device, scored with every model in model_ids, optionally only for
    some of their components); returns its ticket. The pyramid's tensors are kept alive here until it is polled."""
    ids = (_c_i32 * len(model_ids))(*[int(m) for m in model_ids])
    comps = (_c_i32 * len(components))(*[int(c) for c in components]) if components else None
    req = Request(ctypes.pointer(pyramid.desc), ids, len(model_ids), int(form), int(precision), float(tau),
                  comps, len(components) if components else 0)
    t = ctypes.c_uint64()
    _check(lib().tdpm_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    _inflight_requests[(ctx, t.value)] = pyramid
    return t.value


def tdpm_poll(ctx: int, ticket: int, timeout_ms: int = -1, capacity: int = 4096) -> Tuple[np.ndarray, dict]:
    """Wait for a request; returns (detections as DETECTION_DTYPE, info dict). Raises TdpmError(ERR_TIMEOUT) when it
    is not finished within timeout_ms, or the request's own error status when it failed."""
    info = ResultInfo()
    n = ctypes.c_size_t()
    while True:
        out = np.zeros(max(1, capacity), dtype=DETECTION_DTYPE)
        st = lib().tdpm_poll(ctx, int(ticket), int(timeout_ms), out.ctypes.data, int(capacity), ctypes.byref(n),
                             ctypes.byref(info))
        if st == ERR_CAPACITY:
            capacity = int(n.value)
            continue
        break
    if st != ERR_TIMEOUT:
        _inflight_requests.pop((ctx, int(ticket)), None)
    _check(st)
    return out[: n.value], {f: getattr(info, f) for f, _ in ResultInfo._fields_}


def tdpm_detect_thresholds(ctx: int, scores_id: int, tau: np.ndarray, capacity: int = 1 << 20, stream=None,
                           out: Optional[np.ndarray] = None) -> np.ndarray:
    """tdpm_detect with a threshold per (image, component): tau is [n_images][n_components]."""
    t = np.ascontiguousarray(tau, dtype=np.float32)
    if out is None or out.shape[0] < capacity:
        out = np.zeros(capacity, dtype=DETECTION_DTYPE)
    n = ctypes.c_size_t()
    st = lib().tdpm_detect_thresholds(ctx, scores_id, t.ctypes.data, out.ctypes.data if capacity else None,
                                      int(capacity), ctypes.byref(n), _stream_ptr(stream))
    _check(st)
    return out[: n.value]


def tdpm_get_maps(ctx: int, scores_id: int, kind: int, index_a: int, index_b: int, stream=None,
                  image: int = 0) -> np.ndarray:
    """Map (kind, index_a, level index_b) of image `image` of a scores set."""
    rows, cols = _c_i32(), _c_i32()
    st = lib().tdpm_get_maps(ctx, scores_id, kind, image, index_a, index_b, None, 0, ctypes.byref(rows),
                             ctypes.byref(cols), _stream_ptr(stream))
    if st not in (OK, ERR_CAPACITY):
        _check(st)
    if rows.value == 0:
        return np.zeros((0, 0), dtype=np.int32 if kind == MAP_PART_ARG else np.float32)
    out = np.zeros((rows.value, cols.value), dtype=np.int32 if kind == MAP_PART_ARG else np.float32)
    _check(lib().tdpm_get_maps(ctx, scores_id, kind, image, index_a, index_b, out.ctypes.data, out.nbytes,
                               ctypes.byref(rows), ctypes.byref(cols), _stream_ptr(stream)))
    return out


def tdpm_release(ctx: int, scores_id: int) -> None:
    _check(lib().tdpm_release(ctx, scores_id))


# --------------------------------------------------------------------------------------------------- ops
def tdpm_dt_scratch_bytes(H: int, nx: int) -> int:
    return int(lib().tdpm_dt_scratch_bytes(int(H), int(nx)))


def tdpm_dt(S, d: Sequence[float], x_off: int, x_step: int, nx: int, y_off: int, y_step: int, ny: int, D, arg,
            scratch, stream=None) -> None:
    """Distance transform of device map S (torch [H][W] FP32) into D [ny][nx] FP32 and arg [ny][nx] int32."""
    H, W = int(S.shape[0]), int(S.shape[1])
    dd = (ctypes.c_float * 4)(*[float(v) for v in d])
    _check(lib().tdpm_dt(_ptr(S), H, W, dd, x_off, x_step, nx, y_off, y_step, ny, _ptr(D), _ptr(arg), _ptr(scratch),
                         _stream_ptr(stream)))


def tdpm_dt_noalloc_max_elements() -> int:
    return int(lib().tdpm_dt_noalloc_max_elements())


def tdpm_dt_noalloc(S, d: Sequence[float], x_off: int, x_step: int, nx: int, y_off: int, y_step: int, ny: int, D,
                    arg, stream=None) -> None:
    """tdpm_dt without a caller scratch buffer: the library's fixed device scratch is used (no device allocation)."""
    H, W = int(S.shape[0]), int(S.shape[1])
    dd = (ctypes.c_float * 4)(*[float(v) for v in d])
    _check(lib().tdpm_dt_noalloc(_ptr(S), H, W, dd, x_off, x_step, nx, y_off, y_step, ny, _ptr(D), _ptr(arg),
                                 _stream_ptr(stream)))


def tdpm_correlate(feat, filters: np.ndarray, out, precision: int = PREC_FP32, stream=None) -> None:
    """out[k] = correlation of filters[k] ([K][h][w][32] host FP32) with the device level feat ([H][W][32])."""
    f = np.ascontiguousarray(filters, dtype=np.float32)
    K, h, w, _ = f.shape
    _check(lib().tdpm_correlate(_ptr(feat), int(feat.shape[0]), int(feat.shape[1]), f.ctypes.data_as(_c_f32p), K, h, w,
                                int(precision), _ptr(out), _stream_ptr(stream)))


def unpack_arg(a: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Split packed (row << 16) | column argmax values."""
    a = np.asarray(a, dtype=np.int64)
    return (a >> 16).astype(np.int32), (a & 0xFFFF).astype(np.int32)


# --------------------------------------------------------------------------------------------------- instrumentation
def tdpm_kernel_launches() -> int:
    return int(lib().tdpm_kernel_launches())


def tdpm_selftest_bounded_wait(ctx: int) -> int:
    """Run the failure-detection self-test; returns the status it reports (ERR_TIMEOUT when the expiry is seen)."""
    return int(lib().tdpm_selftest_bounded_wait(ctx))


def tdpm_set_fusion(ctx: int, enable: bool = True) -> None:
    """Fused (one kernel) or two-launch channel stage + separable passes of the decomposed per-filter form."""
    _check(lib().tdpm_set_fusion(ctx, 1 if enable else 0))


def tdpm_profile_enable(ctx: int, enable: bool = True) -> None:
    _check(lib().tdpm_profile_enable(ctx, 1 if enable else 0))


def tdpm_profile_read(ctx: int) -> dict:
    """{stage name: (total device ms, launches)} accumulated since the last reset."""
    n = _c_i32()
    _check(lib().tdpm_profile_read(ctx, -1, None, 0, None, None, ctypes.byref(n)))
    out = {}
    for i in range(n.value):
        name = ctypes.create_string_buffer(64)
        ms, cnt = ctypes.c_double(), ctypes.c_int64()
        _check(lib().tdpm_profile_read(ctx, i, name, 64, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(n)))
        out[name.value.decode()] = (ms.value, cnt.value)
    return out


def tdpm_profile_reset(ctx: int) -> None:
    _check(lib().tdpm_profile_reset(ctx))


ZSEP_FORMS = {0: "tile", 1: "persistent/2 stages", 2: "persistent/2 Z buffers", 3: "persistent/2 stages/2 Z buffers",
              4: "persistent"}


def tdpm_autotune_read(ctx: int) -> dict:
    """{shape class: "<N tile width>" or "<N tile width>/persistent", or for the fused decomposed kernel its form}
    picked by the context's autotuner so far."""
    n = _c_i32()
    _check(lib().tdpm_autotune_read(ctx, -1, None, 0, None, None, ctypes.byref(n)))
    out = {}
    for i in range(n.value):
        key = ctypes.create_string_buffer(128)
        nt, pers = _c_i32(), _c_i32()
        _check(lib().tdpm_autotune_read(ctx, i, key, 128, ctypes.byref(nt), ctypes.byref(pers), ctypes.byref(n)))
        k = key.value.decode()
        if k.startswith("zsep:"):
            out[k] = ZSEP_FORMS.get(nt.value, str(nt.value))
        else:
            out[k] = f"{nt.value}/persistent" if pers.value else str(nt.value)
    return out
