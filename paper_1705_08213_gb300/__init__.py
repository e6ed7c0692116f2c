"""Python binding of libccc: the GB300 hot path for 2-way / 3-way CCC.

Argument marshalling only: every function here has the name of a C entry
point declared in ``include/ccc.h`` and forwards torch tensors' device
pointers to it.  Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback.  When the compiled library is missing the
first call raises :class:`CCCError` -- build it with
``paper_1705_08213_gb300.build.build()``.

Genotype panels are torch tensors of shape [n_v, ld] holding the packed
uint64 words (dtype int64 or uint64; the bits are what matter), on the GPU.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "CCCError", "load", "lib_path",
    "CCC_OK", "CCC_EINVAL", "CCC_ERANGE", "CCC_EUNSUPPORTED", "CCC_ECUDA", "CCC_ETIMEOUT",
    "CCC_ENOSPACE", "CCC_EBOUNDS", "CCC_PATH_TC", "CCC_PATH_POPC", "CCC_NORM_PERSNP", "CCC_NORM_JOINT",
    "CCC_OP_METRIC", "CCC_OP_2WAY", "CCC_OP_3WAY", "CCC_MAX_NF",
    "ccc_panel", "ccc_opts", "ccc_opts_default", "ccc_workspace_size", "ccc_allele_counts",
    "ccc2_tally", "ccc2_metric", "ccc2_tally_metric", "ccc3_tally", "ccc3_metric",
    "ccc3_tally_metric", "ccc_status", "ccc2_index", "ccc3_index", "ccc2_count", "ccc3_count",
    "ccc_strerror", "ccc_launch_count", "ccc_timing_enable", "ccc_timing_read",
    "ccc2_tally_metric_noalloc", "ccc_hit", "ccc2_filter", "ccc2_batched_workspace_size",
    "ccc2_batched", "ccc2_batched_tune", "ccc2_tally_metric_rows", "ccc2_rows_count",
    "ccc2_phase_bounds", "ccc2_stream_workspace_size", "ccc2_stream",
    "ccc3_phase_bounds", "ccc3_stream_workspace_size", "ccc3_stream",
    "ccc_panel_multi", "ccc_multi_workspace_size", "ccc_multi_counts", "ccc2_multi_tally",
    "ccc2_multi_tally_metric", "ccc2_multi_metric", "ccc2_multi_tally_metric_rows",
    "ccc2_multi_phase_bounds", "ccc2_multi_stream_workspace_size", "ccc2_multi_stream",
    "ccc_check_bounded_wait", "ccc_checksum",
    "ccc_checked_shrink_outputs",
    "ccc_tune_cache_clear",
    "CCC_MMA_E4M3", "CCC_MMA_E2M1", "CCC_MMA_E2M1_NVF4", "ccc_mma_rate", "ccc_popc_rate",
    "CCC_OPERAND_AUTO", "CCC_OPERAND_E4M3", "CCC_OPERAND_E2M1", "ccc_last_cuda_error",
]

CCC_OK = 0
CCC_EINVAL = -1
CCC_ERANGE = -2
CCC_EUNSUPPORTED = -3
CCC_ECUDA = -4
CCC_ETIMEOUT = -5
CCC_ENOSPACE = -6
CCC_EBOUNDS = -7  # checked build: an index outside its buffer (include/ccc_checked.h)
CCC_PATH_TC = 0
CCC_PATH_POPC = 1
CCC_NORM_PERSNP = 0
CCC_NORM_JOINT = 1
CCC_OP_METRIC = 1
CCC_OP_2WAY = 2
CCC_OP_3WAY = 3
CCC_MAX_NF = 2097151
CCC_MMA_E4M3 = 0
CCC_MMA_E2M1 = 1
CCC_MMA_E2M1_NVF4 = 2
CCC_OPERAND_AUTO = 0
CCC_OPERAND_E4M3 = 1
CCC_OPERAND_E2M1 = 2

# CCC_LIBRARY selects another build of the library (the bounds-checking one,
# paper_1705_08213_gb300/_build_checked/libccc_checked.so, in tests).
lib_path = os.environ.get("CCC_LIBRARY") or _build.LIB


class CCCError(RuntimeError):
    """A libccc call returned a non-zero status (or the library is unavailable)."""

    def __init__(self, name, status):
        self.status = status
        msg = _lib_strerror(status) if isinstance(status, int) else str(status)
        if status == CCC_ECUDA:
            msg += f"; CUDA error {ccc_last_cuda_error()}"
        super().__init__(f"{name}: {msg} ({status})")


class ccc_panel(ctypes.Structure):
    _fields_ = [("geno", ctypes.c_void_p), ("n_f", ctypes.c_int64), ("n_v", ctypes.c_int64),
                ("ld", ctypes.c_int64)]


class ccc_panel_multi(ctypes.Structure):
    _fields_ = [("geno", ctypes.c_void_p), ("n_f", ctypes.c_int64), ("n_v", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("n_states", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ccc_hit(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("j", ctypes.c_int32), ("tally", ctypes.c_int32 * 4),
                ("ccc", ctypes.c_float * 4)]


class ccc_opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("norm", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("group", ctypes.c_int32), ("order", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("split", ctypes.c_int32), ("operand", ctypes.c_int32), ("solo", ctypes.c_int32)]


_lib = None


def load():
    """Load libccc.so (built in-tree).  Raises CCCError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise CCCError("load", f"{lib_path} not built; run paper_1705_08213_gb300.build.build()")
    lib = ctypes.CDLL(lib_path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.ccc_opts_default.argtypes = [P(ccc_opts)]
    lib.ccc_multi_workspace_size.argtypes = [P(ccc_panel_multi), P(ccc_opts), P(ctypes.c_size_t)]
    lib.ccc_multi_counts.argtypes = [P(ccc_panel_multi), vp, vp]
    lib.ccc_check_bounded_wait.argtypes = [vp, i64, vp]
    lib.ccc_checksum.argtypes = [vp, i64, i64, vp, vp]
    lib.ccc2_multi_tally.argtypes = [P(ccc_panel_multi), vp, P(ccc_opts), vp]
    lib.ccc2_multi_tally_metric.argtypes = [P(ccc_panel_multi), vp, vp, P(ccc_opts), vp]
    lib.ccc2_multi_metric.argtypes = [vp, vp, i64, ctypes.c_int32, P(ccc_opts), vp, vp]
    lib.ccc2_multi_tally_metric_rows.argtypes = [P(ccc_panel_multi), i64, i64, vp, vp, P(ccc_opts),
                                                 vp]
    lib.ccc2_multi_phase_bounds.argtypes = [i64, ctypes.c_int32, ctypes.c_int, P(i64)]
    lib.ccc2_multi_stream_workspace_size.argtypes = [P(ccc_panel_multi), ctypes.c_int, P(ccc_opts),
                                                     P(ctypes.c_size_t)]
    lib.ccc2_multi_stream.argtypes = [P(ccc_panel_multi), ctypes.c_int, vp, vp, P(ccc_opts), vp]
    lib.ccc_opts_default.restype = None
    lib.ccc_workspace_size.argtypes = [P(ccc_panel), P(ccc_opts), ctypes.c_int, P(ctypes.c_size_t)]
    lib.ccc_allele_counts.argtypes = [P(ccc_panel), vp, vp]
    lib.ccc2_tally.argtypes = [P(ccc_panel), vp, P(ccc_opts), vp]
    lib.ccc2_metric.argtypes = [vp, vp, i64, P(ccc_opts), vp, vp]
    lib.ccc2_tally_metric.argtypes = [P(ccc_panel), vp, vp, P(ccc_opts), vp]
    lib.ccc3_tally.argtypes = [P(ccc_panel), i64, i64, vp, P(ccc_opts), vp]
    lib.ccc3_metric.argtypes = [vp, vp, i64, i64, i64, P(ccc_opts), vp, vp]
    lib.ccc3_tally_metric.argtypes = [P(ccc_panel), i64, i64, vp, vp, P(ccc_opts), vp]
    lib.ccc_status.argtypes = [P(ccc_opts), P(ctypes.c_int32), vp]
    lib.ccc2_batched_workspace_size.argtypes = [P(ccc_panel), ctypes.c_int, P(ccc_opts),
                                                P(ctypes.c_size_t)]
    lib.ccc2_batched.argtypes = [P(ccc_panel), ctypes.c_int, P(vp), P(vp), P(ccc_opts), vp]
    lib.ccc2_batched_tune.argtypes = [P(ccc_panel), ctypes.c_int, P(vp), P(vp), P(ccc_opts), vp]
    for name in ("ccc2_batched_workspace_size", "ccc2_batched", "ccc2_batched_tune"):
        getattr(lib, name).restype = ctypes.c_int
    lib.ccc2_tally_metric_rows.argtypes = [P(ccc_panel), i64, i64, vp, vp, P(ccc_opts), vp]
    lib.ccc2_tally_metric_rows.restype = ctypes.c_int
    lib.ccc2_rows_count.argtypes = [i64, i64, i64]
    lib.ccc2_rows_count.restype = i64
    lib.ccc2_phase_bounds.argtypes = [i64, ctypes.c_int, P(i64)]
    lib.ccc2_phase_bounds.restype = ctypes.c_int
    lib.ccc2_stream_workspace_size.argtypes = [P(ccc_panel), ctypes.c_int, P(ccc_opts),
                                               P(ctypes.c_size_t)]
    lib.ccc2_stream_workspace_size.restype = ctypes.c_int
    lib.ccc2_stream.argtypes = [P(ccc_panel), ctypes.c_int, vp, vp, P(ccc_opts), vp]
    lib.ccc2_stream.restype = ctypes.c_int
    lib.ccc3_phase_bounds.argtypes = [i64, ctypes.c_int, P(i64)]
    lib.ccc3_phase_bounds.restype = ctypes.c_int
    lib.ccc3_stream_workspace_size.argtypes = [P(ccc_panel), ctypes.c_int, P(ccc_opts),
                                               P(ctypes.c_size_t)]
    lib.ccc3_stream_workspace_size.restype = ctypes.c_int
    lib.ccc3_stream.argtypes = [P(ccc_panel), ctypes.c_int, vp, vp, P(ccc_opts), vp]
    lib.ccc3_stream.restype = ctypes.c_int
    lib.ccc2_filter.argtypes = [P(ccc_panel), ctypes.c_float, vp, i64, vp, P(ccc_opts), vp]
    lib.ccc2_filter.restype = ctypes.c_int
    lib.ccc2_tally_metric_noalloc.argtypes = [P(ccc_panel), vp, vp, vp, P(ccc_opts), vp]
    lib.ccc2_tally_metric_noalloc.restype = ctypes.c_int
    for name in ("ccc_workspace_size", "ccc_allele_counts", "ccc2_tally", "ccc2_metric",
                 "ccc2_tally_metric", "ccc3_tally", "ccc3_metric", "ccc3_tally_metric",
                 "ccc_status"):
        getattr(lib, name).restype = ctypes.c_int
    lib.ccc2_index.argtypes = [i64, i64, i64]
    lib.ccc2_index.restype = i64
    lib.ccc3_index.argtypes = [i64, i64, i64, i64]
    lib.ccc3_index.restype = i64
    lib.ccc2_count.argtypes = [i64]
    lib.ccc2_count.restype = i64
    lib.ccc3_count.argtypes = [i64, i64, i64]
    lib.ccc3_count.restype = i64
    lib.ccc_strerror.argtypes = [ctypes.c_int]
    lib.ccc_strerror.restype = ctypes.c_char_p
    lib.ccc_launch_count.argtypes = []
    lib.ccc_launch_count.restype = ctypes.c_uint64
    lib.ccc_timing_enable.argtypes = [ctypes.c_int]
    lib.ccc_timing_enable.restype = ctypes.c_int
    lib.ccc_timing_read.argtypes = [P(ctypes.c_double), P(ctypes.c_int64)]
    lib.ccc_timing_read.restype = ctypes.c_int
    _lib = lib
    return lib


def _lib_strerror(status):
    try:
        return load().ccc_strerror(status).decode()
    except CCCError:
        return "libccc unavailable"


def _check(name, rc):
    if rc != CCC_OK:
        raise CCCError(name, rc)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _out(name, t, count, width, elem_size=4):
    """Pointer of an output array that must hold count x width elements of elem_size bytes
    (the library writes that many through the raw pointer; a smaller tensor is refused here)."""
    if t is None:
        return None
    if t.numel() * t.element_size() < int(count) * int(width) * elem_size:
        raise CCCError(name, CCC_EINVAL)
    return _ptr(t)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _panel(geno, n_f):
    if geno.dim() != 2 or not geno.is_contiguous() or geno.element_size() != 8:
        raise CCCError("panel", CCC_EINVAL)
    return ccc_panel(geno.data_ptr(), int(n_f), int(geno.shape[0]), int(geno.shape[1]))


def ccc_opts_default(path=CCC_PATH_TC, norm=CCC_NORM_PERSNP, gamma=None, workspace=None, tile=0,
                     operand=CCC_OPERAND_AUTO):
    """A ccc_opts filled by the library's defaults, then by the given fields."""
    o = ccc_opts()
    load().ccc_opts_default(ctypes.byref(o))
    o.path = int(path)
    o.norm = int(norm)
    o.tile = int(tile)
    o.operand = int(operand)
    if gamma is not None:
        o.gamma = float(gamma)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def ccc_workspace_size(geno_or_shape, n_f, opts, op):
    """Workspace bytes for a panel (tensor or (n_v, ld) shape), opts and op."""
    if hasattr(geno_or_shape, "shape") and hasattr(geno_or_shape, "data_ptr"):
        p = _panel(geno_or_shape, n_f)
    else:
        n_v, ld = geno_or_shape
        p = ccc_panel(None, int(n_f), int(n_v), int(ld))
    out = ctypes.c_size_t(0)
    _check("ccc_workspace_size", load().ccc_workspace_size(ctypes.byref(p), ctypes.byref(opts),
                                                           int(op), ctypes.byref(out)))
    return int(out.value)


def ccc_allele_counts(geno, n_f, counts, stream=None):
    p = _panel(geno, n_f)
    _check("ccc_allele_counts", load().ccc_allele_counts(ctypes.byref(p), _ptr(counts), _stream(stream)))


def ccc2_tally(geno, n_f, tally, opts, stream=None):
    p = _panel(geno, n_f)
    n = ccc2_count(p.n_v)
    _check("ccc2_tally", load().ccc2_tally(ctypes.byref(p), _out("ccc2_tally", tally, n, 4),
                                           ctypes.byref(opts), _stream(stream)))


def ccc2_metric(tally, counts, n_v, opts, ccc, stream=None):
    _check("ccc2_metric", load().ccc2_metric(_ptr(tally), _ptr(counts), int(n_v), ctypes.byref(opts),
                                             _ptr(ccc), _stream(stream)))


def _panels(genos, n_fs):
    arr = (ccc_panel * len(genos))()
    for k, (g, n_f) in enumerate(zip(genos, n_fs)):
        arr[k] = _panel(g, n_f)
    return arr


def _ptrs(tensors):
    if tensors is None:
        return None
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def ccc2_batched_workspace_size(genos, n_fs, opts):
    out = ctypes.c_size_t(0)
    arr = _panels(genos, n_fs)
    _check("ccc2_batched_workspace_size",
           load().ccc2_batched_workspace_size(arr, len(genos), ctypes.byref(opts), ctypes.byref(out)))
    return int(out.value)


def ccc2_batched(genos, n_fs, tallies, cccs, opts, stream=None):
    """Batched 2-way: lists of panels (device tensors), their n_f, and output tensors."""
    _check("ccc2_batched", load().ccc2_batched(_panels(genos, n_fs), len(genos), _ptrs(tallies),
                                               _ptrs(cccs), ctypes.byref(opts), _stream(stream)))


def ccc2_batched_tune(genos, n_fs, tallies, cccs, opts, stream=None):
    """Measure the schedule candidates and store the fastest group / order in opts."""
    _check("ccc2_batched_tune", load().ccc2_batched_tune(_panels(genos, n_fs), len(genos),
                                                         _ptrs(tallies), _ptrs(cccs),
                                                         ctypes.byref(opts), _stream(stream)))
    return int(opts.group), int(opts.order)


def ccc2_tally_metric_rows(geno, n_f, i_begin, i_end, tally, ccc, opts, stream=None):
    """2-way over the rows [i_begin, i_end) (one phase)."""
    p = _panel(geno, n_f)
    name = "ccc2_tally_metric_rows"
    n = ccc2_rows_count(p.n_v, max(0, min(int(i_begin), p.n_v)), max(0, min(int(i_end), p.n_v)))
    _check(name, load().ccc2_tally_metric_rows(ctypes.byref(p), int(i_begin), int(i_end),
                                               _out(name, tally, n, 4), _out(name, ccc, n, 4),
                                               ctypes.byref(opts), _stream(stream)))


def ccc2_rows_count(n_v, i_begin, i_end):
    return int(load().ccc2_rows_count(int(n_v), int(i_begin), int(i_end)))


def ccc2_phase_bounds(n_v, n_phases):
    b = (ctypes.c_int64 * (n_phases + 1))()
    _check("ccc2_phase_bounds", load().ccc2_phase_bounds(int(n_v), int(n_phases), b))
    return [int(x) for x in b]


def ccc2_stream_workspace_size(geno_or_shape, n_f, n_phases, opts):
    if hasattr(geno_or_shape, "data_ptr"):
        p = _panel(geno_or_shape, n_f)
    else:
        n_v, ld = geno_or_shape
        p = ccc_panel(None, int(n_f), int(n_v), int(ld))
    out = ctypes.c_size_t(0)
    _check("ccc2_stream_workspace_size",
           load().ccc2_stream_workspace_size(ctypes.byref(p), int(n_phases), ctypes.byref(opts),
                                             ctypes.byref(out)))
    return int(out.value)


def ccc2_stream(geno, n_f, n_phases, host_tally, host_ccc, opts, stream=None):
    """Phased 2-way output into host tensors (pinned for overlap)."""
    p = _panel(geno, n_f)
    _check("ccc2_stream", load().ccc2_stream(ctypes.byref(p), int(n_phases), _ptr(host_tally),
                                             _ptr(host_ccc), ctypes.byref(opts), _stream(stream)))


def ccc3_phase_bounds(n_v, n_phases):
    b = (ctypes.c_int64 * (n_phases + 1))()
    _check("ccc3_phase_bounds", load().ccc3_phase_bounds(int(n_v), int(n_phases), b))
    return [int(x) for x in b]


def ccc3_stream_workspace_size(geno_or_shape, n_f, n_phases, opts):
    if hasattr(geno_or_shape, "data_ptr"):
        p = _panel(geno_or_shape, n_f)
    else:
        n_v, ld = geno_or_shape
        p = ccc_panel(None, int(n_f), int(n_v), int(ld))
    out = ctypes.c_size_t(0)
    _check("ccc3_stream_workspace_size",
           load().ccc3_stream_workspace_size(ctypes.byref(p), int(n_phases), ctypes.byref(opts),
                                             ctypes.byref(out)))
    return int(out.value)


def ccc3_stream(geno, n_f, n_phases, host_tally, host_ccc, opts, stream=None):
    """Phased 3-way output (all triples) into host tensors (pinned for overlap)."""
    p = _panel(geno, n_f)
    _check("ccc3_stream", load().ccc3_stream(ctypes.byref(p), int(n_phases), _ptr(host_tally),
                                             _ptr(host_ccc), ctypes.byref(opts), _stream(stream)))


def ccc2_filter(geno, n_f, threshold, hits, cap, n_hits, opts, stream=None):
    """Thresholded 2-way output: hits is a device buffer of cap ccc_hit records (40 bytes
    each; may be None when cap is 0); n_hits a device int64 tensor receiving the total."""
    p = _panel(geno, n_f)
    _check("ccc2_filter", load().ccc2_filter(ctypes.byref(p), float(threshold),
                                             _out("ccc2_filter", hits, int(cap), 40, 1), int(cap),
                                             _out("ccc2_filter", n_hits, 1, 8, 1),
                                             ctypes.byref(opts), _stream(stream)))


def ccc2_tally_metric(geno, n_f, tally, ccc, opts, stream=None):
    p = _panel(geno, n_f)
    n, name = ccc2_count(p.n_v), "ccc2_tally_metric"
    _check(name, load().ccc2_tally_metric(ctypes.byref(p), _out(name, tally, n, 4),
                                          _out(name, ccc, n, 4), ctypes.byref(opts), _stream(stream)))


def _slab_count(n_v, j_begin, j_end):
    return ccc3_count(n_v, max(0, min(int(j_begin), n_v)), max(0, min(int(j_end), n_v)))


def ccc3_tally(geno, n_f, j_begin, j_end, tally, opts, stream=None):
    p = _panel(geno, n_f)
    n = _slab_count(p.n_v, j_begin, j_end)
    _check("ccc3_tally", load().ccc3_tally(ctypes.byref(p), int(j_begin), int(j_end),
                                           _out("ccc3_tally", tally, n, 8), ctypes.byref(opts),
                                           _stream(stream)))


def ccc3_metric(tally, counts, n_v, j_begin, j_end, opts, ccc, stream=None):
    _check("ccc3_metric", load().ccc3_metric(_ptr(tally), _ptr(counts), int(n_v), int(j_begin),
                                             int(j_end), ctypes.byref(opts), _ptr(ccc),
                                             _stream(stream)))


def ccc3_tally_metric(geno, n_f, j_begin, j_end, tally, ccc, opts, stream=None):
    p = _panel(geno, n_f)
    n, name = _slab_count(p.n_v, j_begin, j_end), "ccc3_tally_metric"
    _check(name, load().ccc3_tally_metric(ctypes.byref(p), int(j_begin), int(j_end),
                                          _out(name, tally, n, 8), _out(name, ccc, n, 8),
                                          ctypes.byref(opts), _stream(stream)))


def ccc_status(opts, stream=None):
    """The workspace status word (synchronises the stream)."""
    st = ctypes.c_int32(0)
    _check("ccc_status", load().ccc_status(ctypes.byref(opts), ctypes.byref(st), _stream(stream)))
    return int(st.value)


def ccc2_index(i, j, n_v):
    return int(load().ccc2_index(int(i), int(j), int(n_v)))


def ccc3_index(i, j, k, n_v):
    return int(load().ccc3_index(int(i), int(j), int(k), int(n_v)))


def ccc2_count(n_v):
    return int(load().ccc2_count(int(n_v)))


def ccc3_count(n_v, j_begin, j_end):
    return int(load().ccc3_count(int(n_v), int(j_begin), int(j_end)))


def ccc_strerror(status):
    return load().ccc_strerror(int(status)).decode()


def ccc_last_cuda_error():
    """The cudaError_t value behind the last CCC_ECUDA of this thread (0 if none)."""
    try:
        lib = load()
    except CCCError:
        return 0
    lib.ccc_last_cuda_error.restype = ctypes.c_int
    return int(lib.ccc_last_cuda_error())


def ccc_launch_count():
    return int(load().ccc_launch_count())


def ccc_timing_enable(enable=True):
    _check("ccc_timing_enable", load().ccc_timing_enable(1 if enable else 0))


def ccc_timing_read():
    """(summed device milliseconds, launches) of the bracketed tally kernels; clears the record."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check("ccc_timing_read", load().ccc_timing_read(ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def ccc2_tally_metric_noalloc(geno, n_f, tally, ccc, opts, status=None, stream=None):
    """Fused 2-way tensor-core call using the library's built-in scratch (no workspace).

    For callers that cannot allocate device memory; ``status`` is an optional
    device int32 tensor that receives the device-side status.
    """
    p = _panel(geno, n_f)
    _check("ccc2_tally_metric_noalloc",
           load().ccc2_tally_metric_noalloc(ctypes.byref(p), _ptr(tally), _ptr(ccc), _ptr(status),
                                            ctypes.byref(opts), _stream(stream)))


# ---------------------------------------------------------------- markers with s states
#
# Multi-allelic panels are torch uint8 tensors of shape [n_v, ld] (one byte per
# entry, x | (y << 4); a nibble >= s marks a missing entry) on the GPU.


def _panel_multi(geno, n_f, s):
    if geno.dim() != 2 or not geno.is_contiguous() or geno.element_size() != 1:
        raise CCCError("panel", CCC_EINVAL)
    return ccc_panel_multi(geno.data_ptr(), int(n_f), int(geno.shape[0]), int(geno.shape[1]),
                           int(s), 0)


def ccc_multi_workspace_size(geno_or_shape, n_f, s, opts):
    """Workspace bytes for a multi-allelic panel (tensor or (n_v, ld) shape) with s states."""
    if hasattr(geno_or_shape, "shape") and hasattr(geno_or_shape, "data_ptr"):
        p = _panel_multi(geno_or_shape, n_f, s)
    else:
        n_v, ld = geno_or_shape
        p = ccc_panel_multi(None, int(n_f), int(n_v), int(ld), int(s), 0)
    out = ctypes.c_size_t(0)
    _check("ccc_multi_workspace_size",
           load().ccc_multi_workspace_size(ctypes.byref(p), ctypes.byref(opts), ctypes.byref(out)))
    return int(out.value)


def ccc_multi_counts(geno, n_f, s, counts, stream=None):
    p = _panel_multi(geno, n_f, s)
    _check("ccc_multi_counts", load().ccc_multi_counts(ctypes.byref(p), _ptr(counts), _stream(stream)))


def ccc2_multi_tally(geno, n_f, s, tally, opts, stream=None):
    p = _panel_multi(geno, n_f, s)
    n = ccc2_count(p.n_v)
    _check("ccc2_multi_tally", load().ccc2_multi_tally(ctypes.byref(p),
                                                       _out("ccc2_multi_tally", tally, n, s * s),
                                                       ctypes.byref(opts), _stream(stream)))


def ccc2_multi_tally_metric(geno, n_f, s, tally, ccc, opts, stream=None):
    p = _panel_multi(geno, n_f, s)
    n, name = ccc2_count(p.n_v), "ccc2_multi_tally_metric"
    _check(name, load().ccc2_multi_tally_metric(ctypes.byref(p), _out(name, tally, n, s * s),
                                                _out(name, ccc, n, s * s), ctypes.byref(opts),
                                                _stream(stream)))


def ccc2_multi_metric(tally, counts, n_v, s, opts, ccc, stream=None):
    _check("ccc2_multi_metric",
           load().ccc2_multi_metric(_ptr(tally), _ptr(counts), int(n_v), int(s), ctypes.byref(opts),
                                    _ptr(ccc), _stream(stream)))


def ccc2_multi_tally_metric_rows(geno, n_f, s, i_begin, i_end, tally, ccc, opts, stream=None):
    p = _panel_multi(geno, n_f, s)
    name = "ccc2_multi_tally_metric_rows"
    n = ccc2_rows_count(p.n_v, max(0, min(int(i_begin), p.n_v)), max(0, min(int(i_end), p.n_v)))
    _check(name, load().ccc2_multi_tally_metric_rows(ctypes.byref(p), int(i_begin), int(i_end),
                                                     _out(name, tally, n, s * s),
                                                     _out(name, ccc, n, s * s), ctypes.byref(opts),
                                                     _stream(stream)))


def ccc2_multi_phase_bounds(n_v, s, n_phases):
    b = (ctypes.c_int64 * (n_phases + 1))()
    _check("ccc2_multi_phase_bounds", load().ccc2_multi_phase_bounds(int(n_v), int(s), int(n_phases), b))
    return list(b)


def ccc2_multi_stream_workspace_size(geno_or_shape, n_f, s, n_phases, opts):
    if hasattr(geno_or_shape, "shape") and hasattr(geno_or_shape, "data_ptr"):
        p = _panel_multi(geno_or_shape, n_f, s)
    else:
        n_v, ld = geno_or_shape
        p = ccc_panel_multi(None, int(n_f), int(n_v), int(ld), int(s), 0)
    out = ctypes.c_size_t(0)
    _check("ccc2_multi_stream_workspace_size",
           load().ccc2_multi_stream_workspace_size(ctypes.byref(p), int(n_phases), ctypes.byref(opts),
                                                   ctypes.byref(out)))
    return int(out.value)


def ccc2_multi_stream(geno, n_f, s, n_phases, host_tally, host_ccc, opts, stream=None):
    p = _panel_multi(geno, n_f, s)
    _check("ccc2_multi_stream",
           load().ccc2_multi_stream(ctypes.byref(p), int(n_phases), _ptr(host_tally), _ptr(host_ccc),
                                    ctypes.byref(opts), _stream(stream)))


def ccc_tune_cache_clear():
    """Forget the batched-schedule choices this process cached (see ccc2_batched_tune)."""
    _check("ccc_tune_cache_clear", load().ccc_tune_cache_clear())


def ccc_checked_shrink_outputs(n):
    """Checked build only (include/ccc_checked.h): later calls tell their kernels that the
    output arrays hold n fewer entries, so the last n stores must be caught (CCC_EBOUNDS)."""
    lib = load()
    lib.ccc_checked_shrink_outputs.argtypes = [ctypes.c_int64]
    _check("ccc_checked_shrink_outputs", lib.ccc_checked_shrink_outputs(int(n)))


def ccc_check_bounded_wait(status, limit_ns, stream=None):
    """Queue the bounded-wait self-test; *status (device int32) receives CCC_ETIMEOUT."""
    _check("ccc_check_bounded_wait", load().ccc_check_bounded_wait(_ptr(status), int(limit_ns),
                                                                   _stream(stream)))


def ccc_checksum(words, base=0, out=None, stream=None):
    """128-bit checksum of a device tensor of 32-bit words (int32 tallies or float32 values)
    whose first word has global index `base`; returns it as a Python int (synchronises)."""
    import torch
    if words.element_size() != 4 or not words.is_contiguous():
        raise CCCError("ccc_checksum", CCC_EINVAL)
    if out is None:
        out = torch.zeros(2, dtype=torch.int64, device=words.device)
    _check("ccc_checksum", load().ccc_checksum(_ptr(words), int(words.numel()), int(base), _ptr(out),
                                               _stream(stream)))
    lo, hi = (int(x) & 0xFFFFFFFFFFFFFFFF for x in out.cpu().tolist())
    return lo | (hi << 64)


def ccc_mma_rate(kind, n_cols=256, n_mma=8192, clusters=None, stream=None):
    """Tensor-core rate probe: (cycles per cluster as a list, bad-entry count).

    `clusters` SM pairs (default: all) each issue n_mma M = 256 x N = n_cols MMAs of the kind
    (CCC_MMA_E4M3, CCC_MMA_E2M1, CCC_MMA_E2M1_NVF4) back to back; synchronises the stream.
    """
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    if clusters is None:
        clusters = torch.cuda.get_device_properties(dev).multi_processor_count // 2
    cycles = torch.zeros(int(clusters), dtype=torch.int64, device=dev)
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    lib = load()
    lib.ccc_mma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    s = _stream(stream)
    _check("ccc_mma_rate", lib.ccc_mma_rate(int(kind), int(n_cols), int(n_mma), int(clusters),
                                            _ptr(cycles), _ptr(bad), s))
    torch.cuda.synchronize(dev)
    return cycles.cpu().tolist(), int(bad.item())


def ccc_popc_rate(iters=4096, blocks=None, stream=None):
    """POPC rate probe: cycles of each 1024-thread block (one block per SM by default)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    if blocks is None:
        blocks = torch.cuda.get_device_properties(dev).multi_processor_count
    cycles = torch.zeros(int(blocks), dtype=torch.int64, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    lib = load()
    lib.ccc_popc_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]
    _check("ccc_popc_rate", lib.ccc_popc_rate(int(iters), int(blocks), _ptr(cycles), _ptr(sink),
                                              _stream(stream)))
    torch.cuda.synchronize(dev)
    return cycles.cpu().tolist()
