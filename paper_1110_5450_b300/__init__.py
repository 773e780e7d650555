"""Python binding of the B300 reconstruction-filter resampler (include/rs.h).

Argument marshalling only: every step of the resampling path (tap indices,
FP64 weight tables, pass kernels) runs in the CUDA kernels of
``librs_b300.so``.  PyTorch is used for device memory and streams.  There is
no CPU fallback: importing this package without the compiled library raises.

The functions keep the C names (``rs_plan_create``, ``rs_resample``,
``rs_plan_recompute``, ``rs_destroy``, ...); ``Plan`` is a small convenience
wrapper that owns one plan and accepts torch tensors.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librs_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "librs_b300.so is not built; run `python paper_1110_5450_b300/build.py` "
        "(the resampler has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------- enums
RS_OK, RS_ERR_INVALID_ARG, RS_ERR_UNSUPPORTED, RS_ERR_OOM, RS_ERR_BUDGET = 0, 1, 2, 3, 4
RS_ERR_CUDA, RS_ERR_TIMEOUT, RS_ERR_BUSY, RS_ERR_DEVICE = 5, 6, 7, 8
RS_F64, RS_F32, RS_F16, RS_BF16 = 0, 1, 2, 3
RS_K_LINEAR, RS_K_CUBIC, RS_K_LANCZOS, RS_K_BSPLINE3, RS_K_MITCHELL, RS_K_GAUSSIAN = 0, 1, 2, 3, 4, 5
RS_B_CLAMP, RS_B_MIRROR, RS_B_REFLECT101, RS_B_TRUNCATE = 0, 1, 2, 3
RS_NO_ANTIALIAS, RS_FORCE_SIMT, RS_FORCE_TC, RS_TWO_PASS, RS_CHECK = 0x1, 0x2, 0x4, 0x8, 0x10
RS_NO_STREAM, RS_FORCE_STREAM, RS_FORCE_VFIRST, RS_PREFILTER = 0x20, 0x40, 0x80, 0x100

KERNELS = {"linear": RS_K_LINEAR, "cubic": RS_K_CUBIC, "lanczos": RS_K_LANCZOS,
           "bspline3": RS_K_BSPLINE3, "mitchell": RS_K_MITCHELL, "gaussian": RS_K_GAUSSIAN}
BOUNDARIES = {"clamp": RS_B_CLAMP, "mirror": RS_B_MIRROR, "reflect101": RS_B_REFLECT101,
              "truncate": RS_B_TRUNCATE}
DEFAULT_PARAM = {"linear": 0.0, "cubic": -0.5, "lanczos": 3.0, "bspline3": 0.0, "mitchell": 1.0 / 3.0,
                 "gaussian": 0.5}
PATHS = {0: "fused", 1: "two_pass", 2: "tcgen05", 3: "stream", 4: "vfirst", 5: "tcstream"}


class rs_plan_desc(ctypes.Structure):
    _fields_ = [("in_h", ctypes.c_int32), ("in_w", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("out_h", ctypes.c_int32), ("out_w", ctypes.c_int32),
                ("scale_h", ctypes.c_double), ("scale_w", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("param", ctypes.c_double),
                ("boundary", ctypes.c_int32),
                ("in_dtype", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
                ("flags", ctypes.c_uint32),
                ("in_row_stride", ctypes.c_int64), ("out_row_stride", ctypes.c_int64)]


class rs_plan_info(ctypes.Structure):
    _fields_ = [("out_h", ctypes.c_int32), ("out_w", ctypes.c_int32),
                ("taps_h", ctypes.c_int32), ("taps_w", ctypes.c_int32),
                ("table_h", ctypes.c_int32), ("table_w", ctypes.c_int32),
                ("path", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("group_h", ctypes.c_int32), ("group_w", ctypes.c_int32),
                ("span_h", ctypes.c_int32), ("span_w", ctypes.c_int32),
                ("warps_pass1", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_int64)]


class rs_stream_form(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("h_warps", ctypes.c_int32), ("staged_blocks", ctypes.c_int32),
                ("strip_width", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("v_warps", ctypes.c_int32), ("row_ranges", ctypes.c_int32)]


class rs_batch_info(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("total_tiles", ctypes.c_int32),
                ("group", ctypes.c_int32), ("warps_pass1", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("use_tma", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("out_pixels", ctypes.c_int64),
                ("in_bytes", ctypes.c_int64), ("out_bytes", ctypes.c_int64), ("n_streamed", ctypes.c_int32)]


class rs_warp_desc(ctypes.Structure):
    _fields_ = [("in_h", ctypes.c_int32), ("in_w", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("out_h", ctypes.c_int32), ("out_w", ctypes.c_int32), ("a", ctypes.c_double * 6),
                ("sigma", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("boundary", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("in_row_stride", ctypes.c_int64), ("out_row_stride", ctypes.c_int64)]


class rs_cluster_desc(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("t_z", ctypes.c_float), ("t_phi", ctypes.c_float),
                ("alpha_z", ctypes.c_float), ("alpha_phi", ctypes.c_float),
                ("max_rounds", ctypes.c_int32)]


class rs_server_desc(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("warps_pass1", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class rs_request(ctypes.Structure):
    _fields_ = [("desc", rs_plan_desc), ("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p)]


class rs_request_state(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("launch_id", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("out_h", ctypes.c_int32), ("out_w", ctypes.c_int32), ("out_row_stride", ctypes.c_int64),
                ("d_out", ctypes.c_void_p), ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64),
                ("t_launch_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64),
                ("t_gpu_start_ns", ctypes.c_uint64), ("t_gpu_end_ns", ctypes.c_uint64)]


class rs_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("completed", "rejected", "launches", "out_pixels", "pending",
                                               "bytes_in_use", "max_bytes_in_use", "max_batch", "streamed",
                                               "launch_host_ns", "stream_host_ns")]


_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)

_lib.rs_desc_out_size.restype = ctypes.c_int
_lib.rs_desc_out_size.argtypes = [ctypes.POINTER(rs_plan_desc), _i32p, _i32p]
_lib.rs_plan_create.restype = ctypes.c_int
_lib.rs_plan_create.argtypes = [ctypes.POINTER(rs_plan_desc), _vp, ctypes.POINTER(_vp)]
_lib.rs_resample.restype = ctypes.c_int
_lib.rs_resample.argtypes = [_vp, _vp, _vp, _vp]
_lib.rs_plan_recompute.restype = ctypes.c_int
_lib.rs_plan_recompute.argtypes = [_vp, _vp]
_lib.rs_destroy.restype = ctypes.c_int
_lib.rs_destroy.argtypes = [_vp]
_lib.rs_plan_get_info.restype = ctypes.c_int
_lib.rs_plan_get_info.argtypes = [_vp, ctypes.POINTER(rs_plan_info)]
_lib.rs_plan_get_tables.restype = ctypes.c_int
_lib.rs_plan_get_tables.argtypes = [_vp, ctypes.c_int, _i32p, _i32p, _i32p, _dp, _dp]
_lib.rs_plan_check.restype = ctypes.c_int
_lib.rs_plan_check.argtypes = [_vp]
_lib.rs_status_string.restype = ctypes.c_char_p
_lib.rs_status_string.argtypes = [ctypes.c_int]
_lib.rs_last_error.restype = ctypes.c_char_p
_lib.rs_last_error.argtypes = []
_lib.rs_version.restype = ctypes.c_int32
_lib.rs_version.argtypes = []
_lib.rs_plan_autotune.restype = ctypes.c_int
_lib.rs_plan_autotune.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_char_p]
_lib.rs_plan_set_stream_form.restype = ctypes.c_int
_lib.rs_plan_set_stream_form.argtypes = [_vp, ctypes.POINTER(rs_stream_form), _vp]
_lib.rs_plan_get_stream_form.restype = ctypes.c_int
_lib.rs_plan_get_stream_form.argtypes = [_vp, ctypes.POINTER(rs_stream_form)]
_lib.rs_plan_set_weights.restype = ctypes.c_int
_lib.rs_plan_set_weights.argtypes = [_vp, ctypes.c_int32, _dp, _vp]
_lib.rs_plan_wait_selftest.restype = ctypes.c_int
_lib.rs_plan_wait_selftest.argtypes = [_vp, ctypes.c_int32, _vp]
_lib.rs_resample_noalloc.restype = ctypes.c_int
_lib.rs_resample_noalloc.argtypes = [ctypes.POINTER(rs_plan_desc), _vp, _vp, _vp]
RS_STATIC_SCRATCH_BYTES = 32 << 20
_vpp = ctypes.POINTER(ctypes.c_void_p)
_lib.rs_batch_create.restype = ctypes.c_int
_lib.rs_batch_create.argtypes = [ctypes.POINTER(rs_plan_desc), ctypes.c_int32, _vp, ctypes.POINTER(_vp)]
_lib.rs_batch_run.restype = ctypes.c_int
_lib.rs_batch_run.argtypes = [_vp, _vpp, _vpp, _vp]
_lib.rs_batch_autotune.restype = ctypes.c_int
_lib.rs_batch_autotune.argtypes = [_vp, _vpp, _vpp, _vp, ctypes.c_char_p]
_lib.rs_batch_get_info.restype = ctypes.c_int
_lib.rs_batch_get_info.argtypes = [_vp, ctypes.POINTER(rs_batch_info)]
_lib.rs_batch_image_path.restype = ctypes.c_int
_lib.rs_batch_image_path.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
_lib.rs_batch_destroy.restype = ctypes.c_int
_lib.rs_batch_destroy.argtypes = [_vp]
_lib.rs_warp.restype = ctypes.c_int
_lib.rs_warp.argtypes = [ctypes.POINTER(rs_warp_desc), _vp, _vp, _vp]
_lib.rs_cluster_create.restype = ctypes.c_int
_lib.rs_cluster_create.argtypes = [ctypes.POINTER(rs_cluster_desc), ctypes.POINTER(_vp)]
_lib.rs_cluster_run.restype = ctypes.c_int
_lib.rs_cluster_run.argtypes = [_vp] * 9 + [_vp]
_lib.rs_cluster_destroy.restype = ctypes.c_int
_lib.rs_cluster_destroy.argtypes = [_vp]
_lib.rs_tc_selftest.restype = ctypes.c_int
_lib.rs_tc_selftest.argtypes = [ctypes.c_int32] * 7 + [_vp, _vp, _vp]
_lib.rs_server_create.restype = ctypes.c_int
_lib.rs_server_create.argtypes = [ctypes.POINTER(rs_server_desc), ctypes.POINTER(_vp)]
_lib.rs_batch_submit.restype = ctypes.c_int
_lib.rs_batch_submit.argtypes = [_vp, ctypes.POINTER(rs_request), ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]
_lib.rs_batch_poll.restype = ctypes.c_int
_lib.rs_batch_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(rs_request_state)]
_lib.rs_server_release.restype = ctypes.c_int
_lib.rs_server_release.argtypes = [_vp, ctypes.c_uint64]
_lib.rs_server_drain.restype = ctypes.c_int
_lib.rs_server_drain.argtypes = [_vp, ctypes.c_int64]
_lib.rs_server_get_stats.restype = ctypes.c_int
_lib.rs_server_get_stats.argtypes = [_vp, ctypes.POINTER(rs_server_stats)]
_lib.rs_server_destroy.restype = ctypes.c_int
_lib.rs_server_destroy.argtypes = [_vp]

# Every symbol include/rs.h declares (checked by the CPU test suite).
EXPORTS = ["rs_desc_out_size", "rs_plan_create", "rs_resample", "rs_plan_recompute", "rs_destroy", "rs_plan_get_info",
           "rs_plan_get_tables", "rs_plan_check", "rs_status_string", "rs_last_error", "rs_version",
           "rs_resample_noalloc", "rs_plan_autotune", "rs_batch_create", "rs_batch_run",
           "rs_batch_autotune", "rs_batch_get_info", "rs_batch_image_path", "rs_batch_destroy", "rs_server_create",
           "rs_batch_submit", "rs_batch_poll", "rs_server_release", "rs_server_drain", "rs_server_get_stats",
           "rs_server_destroy", "rs_tc_selftest", "rs_cluster_create", "rs_cluster_run", "rs_cluster_destroy",
           "rs_warp", "rs_plan_set_stream_form", "rs_plan_get_stream_form", "rs_plan_set_weights",
           "rs_plan_wait_selftest"]


class RSError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = "%s: %s (%s)" % (where, rs_status_string(status), rs_last_error())
        super().__init__(msg)


def _check(status: int, where: str):
    if status != RS_OK:
        raise RSError(status, where)


def rs_status_string(status: int) -> str:
    return _lib.rs_status_string(int(status)).decode()


def rs_last_error() -> str:
    return _lib.rs_last_error().decode()


def rs_version() -> int:
    return int(_lib.rs_version())


def rs_plan_create(desc: rs_plan_desc, stream: int = 0) -> int:
    """Returns the plan handle (an integer); raises RSError on failure."""
    h = _vp()
    _check(_lib.rs_plan_create(ctypes.byref(desc), _vp(stream), ctypes.byref(h)), "rs_plan_create")
    return h.value


def rs_resample(plan: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(_lib.rs_resample(_vp(plan), _vp(d_in), _vp(d_out), _vp(stream)), "rs_resample")


def rs_resample_noalloc(desc: rs_plan_desc, d_in: int, d_out: int, stream: int = 0) -> None:
    """Allocation-free resample through the library's static device scratch
    (for callers that cannot allocate device memory; see include/rs.h)."""
    _check(_lib.rs_resample_noalloc(ctypes.byref(desc), _vp(d_in), _vp(d_out), _vp(stream)),
           "rs_resample_noalloc")


def rs_plan_autotune(plan: int, d_in: int, d_out: int, stream: int = 0, cache_path=None) -> None:
    """Measured autotuning of the fused path on the caller's buffers."""
    cp = None if cache_path is None else os.fsencode(cache_path)
    _check(_lib.rs_plan_autotune(_vp(plan), _vp(d_in), _vp(d_out), _vp(stream), cp), "rs_plan_autotune")


def rs_plan_set_stream_form(plan: int, kind: int, h_warps: int = 0, staged_blocks: int = 0,
                            strip_width: int = 0, prefetch: int = 0, stream: int = 0, v_warps: int = 0,
                            row_ranges: int = 0) -> None:
    """Runs the plan's row-streaming kernel in the given form (0 band kernel,
    phase-alternating; 1 band kernel, warp-specialised; 2 pipelined, with
    `prefetch`, `v_warps` and `row_ranges` options; 3 the tensor-core
    downscale, with `staged_blocks` chunks and `v_warps`)."""
    f = rs_stream_form(int(kind), int(h_warps), int(staged_blocks), int(strip_width), int(prefetch),
                       int(v_warps), int(row_ranges))
    _check(_lib.rs_plan_set_stream_form(_vp(plan), ctypes.byref(f), _vp(stream)), "rs_plan_set_stream_form")


def rs_plan_get_stream_form(plan: int) -> rs_stream_form:
    f = rs_stream_form()
    _check(_lib.rs_plan_get_stream_form(_vp(plan), ctypes.byref(f)), "rs_plan_get_stream_form")
    return f


def rs_plan_recompute(plan: int, stream: int = 0) -> None:
    _check(_lib.rs_plan_recompute(_vp(plan), _vp(stream)), "rs_plan_recompute")


def rs_destroy(plan: int) -> None:
    _check(_lib.rs_destroy(_vp(plan)), "rs_destroy")


def rs_plan_get_info(plan: int) -> rs_plan_info:
    info = rs_plan_info()
    _check(_lib.rs_plan_get_info(_vp(plan), ctypes.byref(info)), "rs_plan_get_info")
    return info


def rs_plan_get_tables(plan: int, axis: int):
    """(jlo, count, start, w64, wwork) numpy arrays of one axis (0 rows, 1 columns)."""
    import numpy as np

    info = rs_plan_get_info(plan)
    n = info.out_h if axis == 0 else info.out_w
    t = info.table_h if axis == 0 else info.table_w
    jlo = np.empty(n, np.int32)
    cnt = np.empty(n, np.int32)
    start = np.empty(n, np.int32)
    w64 = np.empty((n, t), np.float64)
    ww = np.empty((n, t), np.float64)
    _check(_lib.rs_plan_get_tables(_vp(plan), axis, jlo.ctypes.data_as(_i32p), cnt.ctypes.data_as(_i32p),
                                   start.ctypes.data_as(_i32p), w64.ctypes.data_as(_dp),
                                   ww.ctypes.data_as(_dp)), "rs_plan_get_tables")
    return jlo, cnt, start, w64, ww


def rs_plan_check(plan: int) -> None:
    _check(_lib.rs_plan_check(_vp(plan)), "rs_plan_check")


def rs_plan_set_weights(plan: int, axis: int, wwork, stream: int = 0) -> None:
    """Replace one axis' working-precision window weights ((n_out, entries)
    float64 array, as rs_plan_get_tables returns them)."""
    import numpy as np

    w = np.ascontiguousarray(wwork, dtype=np.float64)
    _check(_lib.rs_plan_set_weights(_vp(plan), int(axis), w.ctypes.data_as(_dp), _vp(stream)),
           "rs_plan_set_weights")


def rs_plan_wait_selftest(plan: int, limit_us: int, stream: int = 0) -> None:
    """A bounded device wait that must run out after limit_us (see include/rs.h)."""
    _check(_lib.rs_plan_wait_selftest(_vp(plan), int(limit_us), _vp(stream)), "rs_plan_wait_selftest")


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[int(x) for x in ptrs])
    return arr


def rs_batch_create(descs, stream: int = 0) -> int:
    arr = (rs_plan_desc * len(descs))(*descs)
    h = _vp()
    _check(_lib.rs_batch_create(arr, len(descs), _vp(stream), ctypes.byref(h)), "rs_batch_create")
    return h.value


def rs_batch_run(batch: int, d_in, d_out, stream: int = 0) -> None:
    _check(_lib.rs_batch_run(_vp(batch), _ptr_array(d_in), _ptr_array(d_out), _vp(stream)), "rs_batch_run")


def rs_batch_autotune(batch: int, d_in, d_out, stream: int = 0, cache_path=None) -> None:
    cp = None if cache_path is None else os.fsencode(cache_path)
    _check(_lib.rs_batch_autotune(_vp(batch), _ptr_array(d_in), _ptr_array(d_out), _vp(stream), cp),
           "rs_batch_autotune")


def rs_batch_image_path(batch: int, index: int) -> int:
    """Kernel path of one image of a batch (0 tile, 3 streaming, 5 tensor-core streaming)."""
    v = ctypes.c_int32()
    _check(_lib.rs_batch_image_path(_vp(batch), int(index), ctypes.byref(v)), "rs_batch_image_path")
    return int(v.value)


def rs_batch_get_info(batch: int) -> rs_batch_info:
    info = rs_batch_info()
    _check(_lib.rs_batch_get_info(_vp(batch), ctypes.byref(info)), "rs_batch_get_info")
    return info


def rs_batch_destroy(batch: int) -> None:
    _check(_lib.rs_batch_destroy(_vp(batch)), "rs_batch_destroy")


def rs_tc_selftest(a16, b16, a_mn: int = 0, b_mn: int = 0, variant: int = 0, bf16: int = 1):
    """D = A * B^T on the tensor cores; a16 (m x k) and b16 (n x k) are uint16
    numpy arrays of 16-bit float patterns.  Returns D (m x n float32)."""
    import numpy as np

    a16 = np.ascontiguousarray(a16, dtype=np.uint16)
    b16 = np.ascontiguousarray(b16, dtype=np.uint16)
    m, k = a16.shape
    n = b16.shape[0]
    d = np.zeros((m, n), np.float32)
    _check(_lib.rs_tc_selftest(m, n, k, a_mn, b_mn, variant, bf16, a16.ctypes.data, b16.ctypes.data,
                               d.ctypes.data), "rs_tc_selftest")
    return d


def rs_server_create(budget_bytes: int, max_inflight: int = 4, max_batch: int = 256, warps_pass1: int = 0) -> int:
    d = rs_server_desc(int(budget_bytes), int(max_inflight), int(max_batch), int(warps_pass1), 0)
    h = _vp()
    _check(_lib.rs_server_create(ctypes.byref(d), ctypes.byref(h)), "rs_server_create")
    return h.value


def rs_batch_submit(server: int, reqs) -> int:
    arr = (rs_request * len(reqs))(*reqs)
    t = ctypes.c_uint64()
    _check(_lib.rs_batch_submit(_vp(server), arr, len(reqs), ctypes.byref(t)), "rs_batch_submit")
    return int(t.value)


def rs_batch_poll(server: int, ticket: int) -> rs_request_state:
    st = rs_request_state()
    _check(_lib.rs_batch_poll(_vp(server), ctypes.c_uint64(ticket), ctypes.byref(st)), "rs_batch_poll")
    return st


def rs_server_release(server: int, ticket: int) -> None:
    _check(_lib.rs_server_release(_vp(server), ctypes.c_uint64(ticket)), "rs_server_release")


def rs_server_drain(server: int, timeout_ms: int = 60000) -> None:
    _check(_lib.rs_server_drain(_vp(server), int(timeout_ms)), "rs_server_drain")


def rs_server_get_stats(server: int) -> rs_server_stats:
    st = rs_server_stats()
    _check(_lib.rs_server_get_stats(_vp(server), ctypes.byref(st)), "rs_server_get_stats")
    return st


def rs_server_destroy(server: int) -> None:
    _check(_lib.rs_server_destroy(_vp(server)), "rs_server_destroy")


def rs_desc_out_size(desc: rs_plan_desc):
    """(out_h, out_w) the library derives for a descriptor (host only)."""
    oh, ow = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.rs_desc_out_size(ctypes.byref(desc), ctypes.byref(oh), ctypes.byref(ow)), "rs_desc_out_size")
    return int(oh.value), int(ow.value)


# ------------------------------------------------------------ torch helper
def _torch_dtype_code(dt):
    import torch

    table = {torch.float64: RS_F64, torch.float32: RS_F32, torch.float16: RS_F16,
             torch.bfloat16: RS_BF16}
    if dt not in table:
        raise TypeError("unsupported dtype %s" % dt)
    return table[dt]


def make_desc(in_h, in_w, channels, out_h=0, out_w=0, scale_h=0.0, scale_w=0.0, kernel="lanczos",
              param=None, boundary="mirror", dtype=RS_F32, flags=0, in_row_stride=0,
              out_row_stride=0) -> rs_plan_desc:
    if param is None:
        param = DEFAULT_PARAM[kernel]
    if not isinstance(dtype, int):
        dtype = _torch_dtype_code(dtype)
    return rs_plan_desc(int(in_h), int(in_w), int(channels), int(out_h), int(out_w), float(scale_h),
                        float(scale_w), KERNELS[kernel], float(param), BOUNDARIES[boundary],
                        int(dtype), int(dtype), int(flags), int(in_row_stride), int(out_row_stride))


class Plan:
    """One resampling plan on the current CUDA device.

    >>> p = Plan(4096, 4096, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    >>> y = p(x)          # x: (4096, 4096, 3) float32 CUDA tensor
    """

    def __init__(self, in_h, in_w, channels=1, out_h=0, out_w=0, scale=None, scale_h=None,
                 scale_w=None, kernel="lanczos", param=None, boundary="mirror", dtype=None,
                 flags=0, stream=None):
        import torch

        if dtype is None:
            dtype = torch.float32
        self.torch_dtype = dtype
        sh = scale_h if scale_h is not None else (scale if scale is not None else 0.0)
        sw = scale_w if scale_w is not None else (scale if scale is not None else 0.0)
        self.desc = make_desc(in_h, in_w, channels, out_h, out_w, sh, sw, kernel, param, boundary,
                              _torch_dtype_code(dtype), flags)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.handle = rs_plan_create(self.desc, s.cuda_stream)
        self.info = rs_plan_get_info(self.handle)
        self.in_shape = (int(in_h), int(in_w), int(channels))
        self.out_shape = (self.info.out_h, self.info.out_w, int(channels))

    @property
    def path(self) -> str:
        return PATHS.get(self.info.path, str(self.info.path))

    def __call__(self, x, out=None, stream=None):
        import torch

        if not (x.is_cuda and x.dtype == self.torch_dtype and x.is_contiguous()):
            raise ValueError("input must be a contiguous CUDA tensor of dtype %s" % self.torch_dtype)
        if x.numel() != self.in_shape[0] * self.in_shape[1] * self.in_shape[2]:
            raise ValueError("input has %d elements, plan expects %s" % (x.numel(), self.in_shape))
        if out is None:
            out = torch.empty(self.out_shape, dtype=self.torch_dtype, device=x.device)
        elif not (out.is_cuda and out.dtype == self.torch_dtype and out.is_contiguous()
                  and out.numel() == self.out_shape[0] * self.out_shape[1] * self.out_shape[2]):
            raise ValueError("bad output tensor")
        s = stream if stream is not None else torch.cuda.current_stream()
        rs_resample(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    def autotune(self, x, out=None, stream=None, cache_path=None):
        """Time candidate kernel configurations on (x, out) and keep the fastest."""
        import torch

        if out is None:
            out = torch.empty(self.out_shape, dtype=self.torch_dtype, device=x.device)
        s = stream if stream is not None else torch.cuda.current_stream()
        rs_plan_autotune(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream, cache_path)
        self.info = rs_plan_get_info(self.handle)
        return out

    def recompute(self, stream=None):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        rs_plan_recompute(self.handle, s.cuda_stream)

    def tables(self, axis: int):
        return rs_plan_get_tables(self.handle, axis)

    def check(self):
        rs_plan_check(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            rs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Uneven images resampled by one persistent launch (replayed CUDA graph).

    ``specs``: sequence of dicts with in_h, in_w and either out_h/out_w or
    scale, plus kernel/param/boundary; channels and dtype are batch-wide.
    """

    def __init__(self, specs, channels=1, dtype=None, in_pitches=None, stream=None):
        import torch

        if dtype is None:
            dtype = torch.float32
        self.torch_dtype = dtype
        self.channels = channels
        descs = []
        for i, sp in enumerate(specs):
            sc = sp.get("scale", 0.0)
            pitch = 0 if in_pitches is None else int(in_pitches[i])
            descs.append(make_desc(sp["in_h"], sp["in_w"], channels, sp.get("out_h", 0), sp.get("out_w", 0),
                                   sc, sc, sp.get("kernel", "lanczos"), sp.get("param"),
                                   sp.get("boundary", "mirror"), _torch_dtype_code(dtype),
                                   sp.get("flags", 0), pitch, 0))
        s = stream if stream is not None else torch.cuda.current_stream()
        self.handle = rs_batch_create(descs, s.cuda_stream)
        self.descs = descs
        self.info = rs_batch_get_info(self.handle)

    def __call__(self, ins, outs, stream=None):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        rs_batch_run(self.handle, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], s.cuda_stream)

    def autotune(self, ins, outs, stream=None, cache_path=None):
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        rs_batch_autotune(self.handle, [t.data_ptr() for t in ins], [t.data_ptr() for t in outs], s.cuda_stream,
                          cache_path)
        self.info = rs_batch_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            rs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- affine warps
def rs_warp(desc: rs_warp_desc, d_in, d_out, stream=0):
    _check(_lib.rs_warp(ctypes.byref(desc), d_in, d_out, stream), "rs_warp")


def warp(x, out_h, out_w, a, sigma=0.5, cutoff=3.0, boundary="clamp", out=None, stream=None):
    """Affine warp of an (H, W, C) CUDA tensor with EWA filtering: output
    pixel centre (x + 1/2, y + 1/2) maps to input point
    (a0 x' + a1 y' + a2, a3 x' + a4 y' + a5).  Returns (out_h, out_w, C)."""
    import torch

    if not (x.is_cuda and x.is_contiguous() and x.dim() == 3):
        raise ValueError("input must be a contiguous (H, W, C) CUDA tensor")
    H, W, C = x.shape
    if out is None:
        out = torch.empty((out_h, out_w, C), dtype=x.dtype, device=x.device)
    d = rs_warp_desc(int(H), int(W), int(C), int(out_h), int(out_w), (ctypes.c_double * 6)(*[float(v) for v in a]),
                     float(sigma), float(cutoff), BOUNDARIES[boundary], _torch_dtype_code(x.dtype), 0, 0)
    s = stream if stream is not None else torch.cuda.current_stream()
    rs_warp(d, x.data_ptr(), out.data_ptr(), s.cuda_stream)
    return out


# ---------------------------------------------------------------- clustering
# Table 1 of arXiv:1110.5450 (clustering rows)
CLUSTER_T_Z, CLUSTER_T_PHI = 0.04, 0.009
CLUSTER_ALPHA_Z, CLUSTER_ALPHA_PHI = 8.0 / math.pi, 4.0 / 3.0


def rs_cluster_create(desc: rs_cluster_desc):
    h = _vp()
    _check(_lib.rs_cluster_create(ctypes.byref(desc), ctypes.byref(h)), "rs_cluster_create")
    return h


def rs_cluster_run(handle, z, d, intensity, labels, rounds, region_z=0, region_phi=0, region_size=0, stream=0):
    _check(_lib.rs_cluster_run(handle, z, d, intensity, labels, rounds, region_z or None, region_phi or None,
                               region_size or None, stream), "rs_cluster_run")


def rs_cluster_destroy(handle):
    _check(_lib.rs_cluster_destroy(handle), "rs_cluster_destroy")


class Cluster:
    """The paper's parallel merging clustering of n_frames (height x width)
    ToF frames per call (one thread block per frame).

    >>> c = Cluster(64, 204, 204)
    >>> labels, rounds = c(z, d, intensity)   # (64, 204, 204) float32 CUDA tensors
    """

    def __init__(self, n_frames, height, width, t_z=CLUSTER_T_Z, t_phi=CLUSTER_T_PHI, alpha_z=CLUSTER_ALPHA_Z,
                 alpha_phi=CLUSTER_ALPHA_PHI, max_rounds=0):
        self.shape = (int(n_frames), int(height), int(width))
        self.desc = rs_cluster_desc(int(n_frames), int(height), int(width), float(t_z), float(t_phi),
                                    float(alpha_z), float(alpha_phi), int(max_rounds))
        self.handle = rs_cluster_create(self.desc)

    def __call__(self, z, d, intensity, regions=False, stream=None):
        """Returns (labels int32 (n, h, w), rounds int32 (n,)) and, with
        regions=True, also (mean z, mean phi, pixel count) per region ID."""
        import torch

        for t in (z, d, intensity):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == self.shape):
                raise ValueError("inputs must be contiguous float32 CUDA tensors of shape %s" % (self.shape,))
        dev = z.device
        labels = torch.empty(self.shape, dtype=torch.int32, device=dev)
        rounds = torch.empty(self.shape[0], dtype=torch.int32, device=dev)
        rz = rp = rn = None
        if regions:
            rz = torch.empty(self.shape, dtype=torch.float32, device=dev)
            rp = torch.empty(self.shape, dtype=torch.float32, device=dev)
            rn = torch.empty(self.shape, dtype=torch.int32, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream()
        rs_cluster_run(self.handle, z.data_ptr(), d.data_ptr(), intensity.data_ptr(), labels.data_ptr(),
                       rounds.data_ptr(), rz.data_ptr() if regions else 0, rp.data_ptr() if regions else 0,
                       rn.data_ptr() if regions else 0, s.cuda_stream)
        return (labels, rounds, rz, rp, rn) if regions else (labels, rounds)

    def close(self):
        if getattr(self, "handle", None):
            rs_cluster_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
