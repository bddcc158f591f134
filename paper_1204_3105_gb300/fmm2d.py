"""Thin ctypes binding of libfmm2d (include/fmm2d.h): argument marshalling only.

Every function of the C ABI is exposed under the same name; ``Plan`` wraps a
plan handle.  Device buffers may be given as integers (device pointers) or as
objects with ``data_ptr()`` (e.g. torch CUDA tensors); a stream may be an
integer cudaStream_t, an object with ``cuda_stream``, or None for the legacy
default stream.  The library is loaded from this package directory; if it
has not been built the import of ``lib()`` raises - there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmm2d.so")

QUAD, SEPT, TRI = 0, 1, 2
TILINGS = {"quad": QUAD, "sept": SEPT, "tri": TRI}
PREC_FP64, PREC_MIXED, PREC_MIXED_TC, PREC_HYBRID, PREC_SPLIT = 0x0, 0x1, 0x2, 0x3, 0x4
IN_F32 = 0x10
ADAPTIVE = 0x20
SERVE_PREC_AS_GIVEN = 0x40
FIELD = 0x80

OK, EINVAL, ENOMEM, EDOMAIN, ECUDA, EBUSY, ETIMEOUT, ENOTREADY = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "EDOMAIN", "ECUDA", "EBUSY", "ETIMEOUT", "ENOTREADY"]
STAGES = ["keys", "sort", "tree", "lists", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p", "other",
          "field"]

EXPORTS = {"src_keys": 1, "src_perm": 2, "tgt_keys": 3, "tgt_perm": 4, "cells": 5, "near": 6,
           "far": 7, "multipoles": 8, "locals": 9, "phi_near": 10, "phi_far": 11, "centers": 12,
           "ad_cells": 13, "ad_u": 14, "ad_w": 15, "ad_x": 16, "ad_v": 17}

SYMBOLS = ["fmm2d_default_params", "fmm2d_plan_create", "fmm2d_plan_set_domain", "fmm2d_build",
           "fmm2d_evaluate", "fmm2d_plan_query", "fmm2d_debug_export", "fmm2d_plan_set_profiling",
           "fmm2d_stage_times", "fmm2d_plan_destroy", "fmm2d_last_error",
           "fmm2d_keys_sort_noalloc", "fmm2d_autotune", "fmm2d_measure_alu_peaks",
           "fmm2d_plan_set_params", "fmm2d_serve_create", "fmm2d_serve_submit", "fmm2d_serve_poll",
           "fmm2d_serve_wait", "fmm2d_serve_stats", "fmm2d_serve_destroy",
           "fmm2d_plan_set_leaf_size", "fmm2d_build_forest", "fmm2d_evaluate_field",
           "fmm2d_plan_set_debug_stall", "fmm2d_evaluate_graph"]


class Info(ctypes.Structure):
    _fields_ = [("tiling", ctypes.c_int32), ("levels", ctypes.c_int32), ("p", ctypes.c_int32),
                ("l_min", ctypes.c_int32), ("flags", ctypes.c_uint32), ("built", ctypes.c_int32),
                ("eps", ctypes.c_double), ("domain", ctypes.c_double * 3),
                ("leaf_scale", ctypes.c_double), ("n_src", ctypes.c_int64),
                ("n_tgt", ctypes.c_int64), ("n_cells", ctypes.c_int64 * 24),
                ("n_m2l", ctypes.c_int64), ("n_p2p_pairs", ctypes.c_int64),
                ("n_m2l_ops", ctypes.c_int32), ("max_far", ctypes.c_int32),
                ("max_near", ctypes.c_int32), ("device_error", ctypes.c_int32),
                ("n_leaves", ctypes.c_int64), ("max_leaf_src", ctypes.c_int64),
                ("max_leaf_tgt", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("tiling", ctypes.c_int32), ("levels", ctypes.c_int32), ("p", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("eps", ctypes.c_double), ("domain", ctypes.c_double * 3),
                ("src_xy", ctypes.c_void_p), ("n_src", ctypes.c_int64), ("tgt_xy", ctypes.c_void_p),
                ("n_tgt", ctypes.c_int64), ("strengths", ctypes.c_void_p),
                ("potentials", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("levels", ctypes.c_int32), ("p", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("slot", ctypes.c_int32), ("batched", ctypes.c_int32),
                ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("error", ctypes.c_char * 128)]


class ServeInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("slots", ctypes.c_int32)]


class FMM2DError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


_LIB = None


def lib():
    """Load libfmm2d.so (raises if it is missing) and declare its signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfmm2d.so is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.fmm2d_default_params.argtypes = [c_int, i64, c_int, dbl, ctypes.POINTER(c_int),
                                       ctypes.POINTER(c_int), ctypes.POINTER(dbl)]
    L.fmm2d_plan_create.argtypes = [c_int, c_int, c_int, dbl, ctypes.c_uint, ctypes.POINTER(vp)]
    L.fmm2d_plan_set_domain.argtypes = [vp, dbl, dbl, dbl]
    L.fmm2d_build.argtypes = [vp, vp, i64, vp, i64, vp]
    L.fmm2d_evaluate.argtypes = [vp, vp, vp, vp]
    L.fmm2d_evaluate_graph.argtypes = [vp, vp, vp, vp]
    L.fmm2d_evaluate_field.argtypes = [vp, vp, vp, vp, vp]
    L.fmm2d_plan_query.argtypes = [vp, ctypes.POINTER(Info)]
    L.fmm2d_debug_export.argtypes = [vp, c_int, c_int, vp, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_size_t)]
    L.fmm2d_plan_set_profiling.argtypes = [vp, c_int]
    L.fmm2d_plan_set_debug_stall.argtypes = [vp, c_int]
    L.fmm2d_stage_times.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64), c_int,
                                    ctypes.POINTER(c_int)]
    L.fmm2d_plan_destroy.argtypes = [vp]
    L.fmm2d_plan_destroy.restype = None
    L.fmm2d_last_error.argtypes = [vp]
    L.fmm2d_last_error.restype = ctypes.c_char_p
    L.fmm2d_keys_sort_noalloc.argtypes = [c_int, c_int, dbl, ctypes.POINTER(dbl), vp, i64,
                                          ctypes.c_uint, vp, vp, vp, ctypes.c_char_p,
                                          ctypes.c_size_t]
    L.fmm2d_autotune.argtypes = [c_int, dbl, ctypes.c_uint, ctypes.POINTER(dbl), vp, i64, vp, i64,
                                 vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                 ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.fmm2d_measure_alu_peaks.argtypes = [ctypes.POINTER(dbl)]
    L.fmm2d_plan_set_params.argtypes = [vp, c_int, c_int, dbl]
    L.fmm2d_plan_set_leaf_size.argtypes = [vp, c_int]
    L.fmm2d_build_forest.argtypes = [vp, vp, ctypes.POINTER(i64), c_int, vp]
    L.fmm2d_serve_create.argtypes = [ctypes.c_size_t, c_int, ctypes.POINTER(vp)]
    L.fmm2d_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.fmm2d_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    L.fmm2d_serve_wait.argtypes = [vp, ctypes.c_uint64, dbl, ctypes.POINTER(Result)]
    L.fmm2d_serve_stats.argtypes = [vp, ctypes.POINTER(ServeInfo)]
    L.fmm2d_serve_destroy.argtypes = [vp]
    L.fmm2d_serve_destroy.restype = None
    for name in SYMBOLS:
        if name not in ("fmm2d_plan_destroy", "fmm2d_last_error", "fmm2d_serve_destroy"):
            getattr(L, name).restype = c_int
    _LIB = L
    return L


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def fmm2d_default_params(tiling, n_points, leaf_target=64, eps=1e-6):
    L, p = ctypes.c_int(), ctypes.c_int()
    r = ctypes.c_double()
    st = lib().fmm2d_default_params(TILINGS.get(tiling, tiling), int(n_points), int(leaf_target),
                                    float(eps), ctypes.byref(L), ctypes.byref(p), ctypes.byref(r))
    if st:
        raise FMM2DError(st, "fmm2d_default_params")
    return L.value, p.value, r.value


def fmm2d_keys_sort_noalloc(tiling, levels, leaf_scale, domain, xy, n, flags, keys_out,
                            perm_out, stream=None):
    """Leaf keys and stable sort permutation without any GPU allocation (see
    include/fmm2d.h); keys_out / perm_out are caller-owned n-element uint32
    (or int32) device buffers."""
    buf = ctypes.create_string_buffer(256)
    dom = None if domain is None else (ctypes.c_double * 3)(*domain)
    st = lib().fmm2d_keys_sort_noalloc(TILINGS.get(tiling, tiling), int(levels), float(leaf_scale),
                                       dom, _ptr(xy), int(n), int(flags), _ptr(keys_out),
                                       _ptr(perm_out), _stream(stream), buf, 256)
    if st:
        raise FMM2DError(st, buf.value.decode())


def fmm2d_autotune(tiling, eps, flags, src_xy, n_src, tgt_xy, n_tgt, domain=None, stream=None):
    """Measured choice of (L, p); returns (levels, p, err, ms) (see include/fmm2d.h)."""
    L, p = ctypes.c_int(), ctypes.c_int()
    err, ms = ctypes.c_double(), ctypes.c_double()
    dom = None if domain is None else (ctypes.c_double * 3)(*domain)
    st = lib().fmm2d_autotune(TILINGS.get(tiling, tiling), float(eps), int(flags), dom, _ptr(src_xy),
                              int(n_src), _ptr(tgt_xy), int(n_tgt), _stream(stream), ctypes.byref(L),
                              ctypes.byref(p), ctypes.byref(err), ctypes.byref(ms))
    if st:
        raise FMM2DError(st, "fmm2d_autotune")
    return L.value, p.value, err.value, ms.value


def fmm2d_measure_alu_peaks():
    """{"fp32_tflops", "lg2_gops", "fp64_tflops", "sms", "tf32_tflops"} measured on the
    current device."""
    out = (ctypes.c_double * 5)()
    st = lib().fmm2d_measure_alu_peaks(out)
    if st:
        raise FMM2DError(st, "fmm2d_measure_alu_peaks")
    return {"fp32_tflops": out[0], "lg2_gops": out[1], "fp64_tflops": out[2], "sms": int(out[3]),
            "tf32_tflops": out[4]}


class Plan:
    """A plan handle: ``fmm2d_plan_create`` on construction,
    ``fmm2d_plan_destroy`` on ``close``."""

    def __init__(self, tiling, levels=0, p=0, eps=1e-6, flags=PREC_MIXED):
        self._h = ctypes.c_void_p()
        self.lib = lib()
        st = self.lib.fmm2d_plan_create(TILINGS.get(tiling, tiling), int(levels), int(p),
                                        float(eps), int(flags), ctypes.byref(self._h))
        if st:
            raise FMM2DError(st, self.lib.fmm2d_last_error(None).decode())
        self.flags = flags

    def _check(self, st, what):
        if st:
            raise FMM2DError(st, "%s: %s" % (what, self.lib.fmm2d_last_error(self._h).decode()))

    def fmm2d_plan_set_leaf_size(self, leaf_size):
        self._check(self.lib.fmm2d_plan_set_leaf_size(self._h, int(leaf_size)), "set_leaf_size")

    set_leaf_size = fmm2d_plan_set_leaf_size

    def fmm2d_plan_set_domain(self, x0, y0, size):
        self._check(self.lib.fmm2d_plan_set_domain(self._h, float(x0), float(y0), float(size)),
                    "set_domain")

    set_domain = fmm2d_plan_set_domain

    def fmm2d_build(self, src_xy, n_src, tgt_xy, n_tgt, stream=None):
        self._check(self.lib.fmm2d_build(self._h, _ptr(src_xy), int(n_src), _ptr(tgt_xy),
                                         int(n_tgt), _stream(stream)), "build")

    build = fmm2d_build

    def fmm2d_build_forest(self, xy, offsets, stream=None):
        """xy: device points of all instances; offsets: host int64 array, n_inst + 1 entries."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self._check(self.lib.fmm2d_build_forest(
            self._h, _ptr(xy), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1,
            _stream(stream)), "build_forest")

    build_forest = fmm2d_build_forest

    def fmm2d_evaluate(self, strengths, potentials, stream=None):
        self._check(self.lib.fmm2d_evaluate(self._h, _ptr(strengths), _ptr(potentials),
                                            _stream(stream)), "evaluate")

    evaluate = fmm2d_evaluate

    def fmm2d_evaluate_graph(self, strengths, potentials, stream=None):
        """fmm2d_evaluate replayed from a recorded CUDA graph (same pointers)."""
        self._check(self.lib.fmm2d_evaluate_graph(self._h, _ptr(strengths), _ptr(potentials),
                                                  _stream(stream)), "evaluate_graph")

    evaluate_graph = fmm2d_evaluate_graph

    def fmm2d_evaluate_field(self, strengths, potentials, field, stream=None):
        """field: 2 * n_tgt float64 device values (Re F, Im F) per target."""
        self._check(self.lib.fmm2d_evaluate_field(self._h, _ptr(strengths), _ptr(potentials),
                                                  _ptr(field), _stream(stream)), "evaluate_field")

    evaluate_field = fmm2d_evaluate_field

    def fmm2d_plan_query(self):
        info = Info()
        self._check(self.lib.fmm2d_plan_query(self._h, ctypes.byref(info)), "query")
        d = {f: getattr(info, f) for f, _ in Info._fields_}
        d["domain"] = list(info.domain)
        d["n_cells"] = list(info.n_cells)[: max(0, info.levels) + 1]
        return d

    query = fmm2d_plan_query

    def fmm2d_debug_export(self, what, level=0):
        w = EXPORTS.get(what, what)
        n = ctypes.c_size_t()
        self._check(self.lib.fmm2d_debug_export(self._h, w, int(level), None, 0, ctypes.byref(n)),
                    "export")
        buf = np.zeros(max(1, n.value), np.uint8)
        self._check(self.lib.fmm2d_debug_export(self._h, w, int(level), buf.ctypes.data, buf.nbytes,
                                                ctypes.byref(n)), "export")
        buf = buf[: n.value]
        if w in (1, 2, 3, 4, 5):
            return buf.view(np.int64)
        if w in (6, 7):
            return buf.view(np.int64).reshape(-1, 2)
        if w in (8, 9):
            p = self.query()["p"]
            return buf.view(np.complex128).reshape(-1, p + 1)
        if w == 12:
            return buf.view(np.complex128)
        if w == 13:
            return buf.view(np.int64).reshape(-1, 3)
        if w in (14, 15, 16, 17):
            return buf.view(np.int64).reshape(-1, 4)
        return buf.view(np.float64)

    export = fmm2d_debug_export

    def fmm2d_plan_set_profiling(self, on=True):
        """on: False/0 off, True/1 stage events, 2 stage events with the stages serialised."""
        self._check(self.lib.fmm2d_plan_set_profiling(self._h, int(on)), "profiling")

    set_profiling = fmm2d_plan_set_profiling

    def fmm2d_plan_set_debug_stall(self, on=True):
        """Test switch: tensor-core M2L CTAs time out before their MMAs."""
        self._check(self.lib.fmm2d_plan_set_debug_stall(self._h, int(on)), "debug_stall")

    set_debug_stall = fmm2d_plan_set_debug_stall

    def fmm2d_stage_times(self):
        ms = (ctypes.c_double * 16)()
        ln = (ctypes.c_int64 * 16)()
        n = ctypes.c_int()
        self._check(self.lib.fmm2d_stage_times(self._h, ms, ln, 16, ctypes.byref(n)), "stage_times")
        return {STAGES[i]: (ms[i], ln[i]) for i in range(min(n.value, len(STAGES)))}

    stage_times = fmm2d_stage_times

    def close(self):
        if self._h:
            self.lib.fmm2d_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(a):
    """Address of a C-contiguous numpy array (host memory)."""
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return a.ctypes.data


class Server:
    """fmm2d_serve_* wrapper.  Inputs and outputs are host numpy arrays that
    the caller keeps alive until the request completes."""

    def __init__(self, hbm_budget_bytes, max_slots=8):
        self.lib = lib()
        self._h = ctypes.c_void_p()
        st = self.lib.fmm2d_serve_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(self._h))
        if st:
            raise FMM2DError(st, "fmm2d_serve_create")
        self._keep = {}

    def fmm2d_serve_submit(self, tiling, src_xy, strengths, potentials, tgt_xy=None, eps=1e-6,
                           levels=0, p=0, flags=0, domain=None):
        f32 = src_xy.dtype == np.float32
        r = Request()
        r.tiling = TILINGS.get(tiling, tiling)
        r.levels, r.p = int(levels), int(p)
        r.flags = int(flags) | (IN_F32 if f32 else 0)
        r.eps = float(eps)
        r.domain[:] = list(domain) if domain is not None else [0.0, 0.0, 0.0]
        r.src_xy, r.n_src = _host_ptr(src_xy), len(src_xy)
        r.tgt_xy = _host_ptr(tgt_xy)
        r.n_tgt = 0 if tgt_xy is None else len(tgt_xy)
        r.strengths, r.potentials = _host_ptr(strengths), _host_ptr(potentials)
        t = ctypes.c_uint64()
        st = self.lib.fmm2d_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        if st:
            raise FMM2DError(st, "fmm2d_serve_submit")
        self._keep[t.value] = (src_xy, strengths, potentials, tgt_xy)
        return t.value

    submit = fmm2d_serve_submit

    def _result(self, t, res):
        self._keep.pop(t, None)
        d = {f: getattr(res, f) for f, _ in Result._fields_}
        d["error"] = res.error.decode(errors="replace")
        return d

    def fmm2d_serve_poll(self, ticket):
        res = Result()
        st = self.lib.fmm2d_serve_poll(self._h, int(ticket), ctypes.byref(res))
        if st == ENOTREADY:
            return None
        if st:
            raise FMM2DError(st, "fmm2d_serve_poll")
        return self._result(ticket, res)

    poll = fmm2d_serve_poll

    def fmm2d_serve_wait(self, ticket, timeout_ms=60000.0):
        res = Result()
        st = self.lib.fmm2d_serve_wait(self._h, int(ticket), float(timeout_ms), ctypes.byref(res))
        if st:
            raise FMM2DError(st, "fmm2d_serve_wait")
        return self._result(ticket, res)

    wait = fmm2d_serve_wait

    def fmm2d_serve_stats(self):
        info = ServeInfo()
        self.lib.fmm2d_serve_stats(self._h, ctypes.byref(info))
        return {f: getattr(info, f) for f, _ in ServeInfo._fields_}

    stats = fmm2d_serve_stats

    def close(self):
        if self._h:
            self.lib.fmm2d_serve_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
