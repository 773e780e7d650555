"""FP64 CPU oracle for separable image resampling with reconstruction filters.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs import this
package.  The product package (``paper_1110_5450_b300``) never imports it, and
the two share no code, header, table or constant.

The arithmetic lives in ``rs_oracle.c`` (plain C, double precision, a direct
two-dimensional summation threaded over output rows); this module compiles it
with gcc and wraps it with ctypes.  ``brute`` holds an exact-rational
brute force for tiny grids, written independently from the coordinate
definitions.

Conventions (standard definitions; the paper itself states no resampling
formula, so each is cited to its published source in ``rs_oracle.c``):
half-pixel centres, kernel widened by max(1, n_in/n_out) when downsampling,
strict support |x| < R, weights normalised to sum 1, boundary maps clamp /
mirror (half-sample symmetric) / reflect101 / truncate.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KERNELS = {"linear": 0, "cubic": 1, "lanczos": 2, "bspline3": 3, "mitchell": 4, "gaussian": 5}
BOUNDARIES = {"clamp": 0, "mirror": 1, "reflect101": 2, "truncate": 3}
DEFAULT_PARAM = {"linear": 0.0, "cubic": -0.5, "lanczos": 3.0, "bspline3": 0.0, "mitchell": 1.0 / 3.0,
                 "gaussian": 0.5}

_lock = threading.Lock()
_default = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle C source into a shared library (gcc -O2, no FP
    contraction).  ``src``/``out`` let tests build a deliberately broken copy."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
             "-Wall", "-o", tmp, src, "-lpthread", "-lm"]
        )
        os.replace(tmp, out)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i64, dbl, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    p64 = ctypes.POINTER(ctypes.c_int64)
    pd = ctypes.POINTER(ctypes.c_double)
    lib.ora_kernel_value.restype = dbl
    lib.ora_kernel_value.argtypes = [ip, dbl, dbl]
    lib.ora_axis_taps.restype = ip
    lib.ora_axis_taps.argtypes = [i64, i64, ip, dbl, ip, i64, p64, p64]
    lib.ora_boundary_map.restype = i64
    lib.ora_boundary_map.argtypes = [i64, i64, ip]
    lib.ora_axis_weights.restype = ip
    lib.ora_axis_weights.argtypes = [i64, i64, ip, dbl, ip, ip, i64, i64, p64, p64, p64, pd]
    lib.ora_resample_rows.restype = ip
    lib.ora_resample_rows.argtypes = [ctypes.c_void_p, i64, i64, i64, i64, i64, ip, dbl,
                                      ip, ip, i64, i64, ctypes.c_void_p, ip]
    lib.ora_default_threads.restype = ip
    lib.ora_default_threads.argtypes = []
    return lib


def _kp(kernel: str, param):
    if param is None:
        param = DEFAULT_PARAM[kernel]
    return KERNELS[kernel], float(param)


class Oracle:
    """One loaded copy of the oracle library (the default one, or a test's
    deliberately broken copy)."""

    def __init__(self, path: str):
        self.path = path
        self.lib = _bind(path)

    def default_threads(self) -> int:
        return int(self.lib.ora_default_threads())

    def kernel_value(self, kernel: str, x: float, param=None) -> float:
        k, p = _kp(kernel, param)
        return float(self.lib.ora_kernel_value(k, p, float(x)))

    def boundary_map(self, j: int, n: int, boundary: str) -> int:
        return int(self.lib.ora_boundary_map(int(j), int(n), BOUNDARIES[boundary]))

    def axis_taps(self, n_in: int, n_out: int, kernel: str, i: int, param=None, antialias=True):
        """(j_first, count) of output i: raw (unmapped) consecutive taps."""
        k, p = _kp(kernel, param)
        jf, cnt = ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.ora_axis_taps(n_in, n_out, k, p, int(bool(antialias)), i,
                                    ctypes.byref(jf), ctypes.byref(cnt))
        if rc:
            raise ValueError("ora_axis_taps failed: %d" % rc)
        return int(jf.value), int(cnt.value)

    def axis_weights(self, n_in: int, n_out: int, kernel: str, boundary: str, param=None,
                     antialias=True):
        """Per output i: (j_first, mapped index array, normalised FP64 weights)."""
        k, p = _kp(kernel, param)
        cap = 4 * (n_in // max(1, n_out) + 2) * 16 + 64
        rows = []
        idx = (ctypes.c_int64 * cap)()
        w = (ctypes.c_double * cap)()
        jf, cnt = ctypes.c_int64(), ctypes.c_int64()
        for i in range(n_out):
            rc = self.lib.ora_axis_weights(n_in, n_out, k, p, BOUNDARIES[boundary],
                                           int(bool(antialias)), i, cap, ctypes.byref(jf),
                                           ctypes.byref(cnt), idx, w)
            if rc:
                raise ValueError("ora_axis_weights failed: %d" % rc)
            n = cnt.value
            rows.append((int(jf.value), np.array(idx[:n], dtype=np.int64),
                         np.array(w[:n], dtype=np.float64)))
        return rows

    def axis_weights_at(self, n_in: int, n_out: int, kernel: str, boundary: str, i: int, param=None,
                        antialias=True):
        """(j_first, mapped index array, normalised FP64 weights) of output i
        alone (for sampled outputs of long axes)."""
        k, p = _kp(kernel, param)
        cap = 4 * (n_in // max(1, n_out) + 2) * 16 + 64
        idx = (ctypes.c_int64 * cap)()
        w = (ctypes.c_double * cap)()
        jf, cnt = ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.ora_axis_weights(n_in, n_out, k, p, BOUNDARIES[boundary], int(bool(antialias)), i, cap,
                                       ctypes.byref(jf), ctypes.byref(cnt), idx, w)
        if rc:
            raise ValueError("ora_axis_weights failed: %d" % rc)
        n = cnt.value
        return int(jf.value), np.array(idx[:n], dtype=np.int64), np.array(w[:n], dtype=np.float64)

    def bspline_matrix(self, n: int, boundary: str) -> np.ndarray:
        """n x n matrix of the cubic B-spline interpolation condition on one
        axis (M. Unser, IEEE SP Mag. 16(6), 1999): sample k equals
        sum_j beta3(k - j) c[B(j)] over the integers j, the coefficients c
        extended by the boundary map B."""
        M = np.zeros((n, n))
        for k in range(n):
            for j in range(k - 2, k + 3):
                M[k, self.boundary_map(j, n, boundary)] += self.kernel_value("bspline3", float(k - j))
        return M

    def bspline_coefficients(self, img, boundary: str) -> np.ndarray:
        """Cubic B-spline coefficients of an (H, W) or (H, W, C) image: the
        interpolation condition solved along the columns, then the rows."""
        a = np.asarray(img, dtype=np.float64)
        squeeze = a.ndim == 2
        if squeeze:
            a = a[:, :, None]
        H, W, C = a.shape
        Mh, Mw = self.bspline_matrix(H, boundary), self.bspline_matrix(W, boundary)
        c = np.linalg.solve(Mh, a.reshape(H, W * C)).reshape(H, W, C)
        c = np.linalg.solve(Mw, c.transpose(1, 0, 2).reshape(W, H * C)).reshape(W, H, C).transpose(1, 0, 2)
        c = np.ascontiguousarray(c)
        return c[:, :, 0] if squeeze else c

    def resample(self, img, out_h: int, out_w: int, kernel: str, boundary: str, param=None,
                 antialias: bool = True, rows=None, nthreads: int = 0, prefilter: bool = False) -> np.ndarray:
        """Resample an (H, W) or (H, W, C) image in FP64.

        ``rows=(y0, y1)`` computes only output rows [y0, y1) (used to time a
        bounded sample).  The input is converted to float64 exactly.  With
        ``prefilter`` (cubic B-spline only) the image is first replaced by its
        B-spline coefficients, which makes the B-spline interpolating.
        """
        if prefilter:
            if kernel != "bspline3":
                raise ValueError("prefilter applies to the cubic B-spline")
            img = self.bspline_coefficients(img, boundary)
        a = np.asarray(img)
        squeeze = a.ndim == 2
        if squeeze:
            a = a[:, :, None]
        if a.ndim != 3:
            raise ValueError("image must be (H, W) or (H, W, C)")
        a = np.ascontiguousarray(a, dtype=np.float64)
        H, W, C = a.shape
        y0, y1 = (0, out_h) if rows is None else rows
        out = np.empty((y1 - y0, out_w, C), dtype=np.float64)
        k, p = _kp(kernel, param)
        rc = self.lib.ora_resample_rows(a.ctypes.data, H, W, C, out_h, out_w, k, p,
                                        BOUNDARIES[boundary], int(bool(antialias)), y0, y1,
                                        out.ctypes.data, int(nthreads))
        if rc:
            raise ValueError("ora_resample_rows failed: %d" % rc)
        return out[:, :, 0] if squeeze else out


def default() -> Oracle:
    """The oracle built from ``rs_oracle.c`` (compiled on first use)."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def out_size(n: int, scale: float) -> int:
    """Output length for a scale factor: max(1, floor(n * scale + 1/2))."""
    return max(1, int(math.floor(n * scale + 0.5)))


def default_threads() -> int:
    return default().default_threads()


def kernel_value(kernel: str, x: float, param=None) -> float:
    return default().kernel_value(kernel, x, param)


def boundary_map(j: int, n: int, boundary: str) -> int:
    return default().boundary_map(j, n, boundary)


def axis_taps(n_in: int, n_out: int, kernel: str, i: int, param=None, antialias=True):
    return default().axis_taps(n_in, n_out, kernel, i, param, antialias)


def axis_weights(n_in: int, n_out: int, kernel: str, boundary: str, param=None, antialias=True):
    return default().axis_weights(n_in, n_out, kernel, boundary, param, antialias)


def axis_weights_at(n_in: int, n_out: int, kernel: str, boundary: str, i: int, param=None, antialias=True):
    return default().axis_weights_at(n_in, n_out, kernel, boundary, i, param, antialias)


def resample(img, out_h: int, out_w: int, kernel: str, boundary: str, param=None,
             antialias: bool = True, rows=None, nthreads: int = 0, prefilter: bool = False) -> np.ndarray:
    return default().resample(img, out_h, out_w, kernel, boundary, param, antialias, rows,
                              nthreads, prefilter)


def bspline_coefficients(img, boundary: str) -> np.ndarray:
    return default().bspline_coefficients(img, boundary)
