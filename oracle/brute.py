"""Exact-rational brute force for tiny grids (TEST INFRASTRUCTURE ONLY).

Written straight from the coordinate definitions, independently of
``rs_oracle.c``: output sample i of an axis sits at c_i = (i + 1/2) n_in / n_out
(half-pixel centres), input sample j at j + 1/2, the kernel is widened by
sc = max(1, n_in / n_out) when antialiasing, and tap j belongs to output i
when |j + 1/2 - c_i| / sc < R.  All of this is done in ``fractions.Fraction``,
so the tap sets are exact.  Polynomial kernels (linear, Keys cubic, cubic
B-spline, Mitchell-Netravali) are evaluated exactly as well; Lanczos and the
Gaussian fall back to float math.

The result is the dense resampling matrix M (n_out x n_in) of one axis, with
the boundary map folded in; a 2-D image resamples as M_h @ X @ M_w^T per
channel.  Pure Python: use on grids of a few dozen samples at most.
"""
from __future__ import annotations

import functools
import math
from fractions import Fraction

SUPPORT = {"linear": 1, "cubic": 2, "bspline3": 2, "mitchell": 2}


def support(kernel: str, param) -> int:
    if kernel == "lanczos":
        return int(param)
    if kernel == "gaussian":
        return math.ceil(3 * param)
    return SUPPORT[kernel]


def kernel_exact(kernel: str, x: Fraction, param):
    """K(x) exactly for polynomial kernels (Fraction), float for Lanczos."""
    t = abs(x)
    if kernel == "linear":
        return 1 - t if t < 1 else Fraction(0)
    if kernel == "cubic":
        a = Fraction(param)
        if t < 1:
            return (a + 2) * t ** 3 - (a + 3) * t ** 2 + 1
        if t < 2:
            return a * t ** 3 - 5 * a * t ** 2 + 8 * a * t - 4 * a
        return Fraction(0)
    if kernel == "bspline3":
        if t < 1:
            return Fraction(2, 3) - t ** 2 + t ** 3 / 2
        if t < 2:
            return (2 - t) ** 3 / 6
        return Fraction(0)
    if kernel == "mitchell":
        # Mitchell & Netravali (1988) with C = (1 - B) / 2, exact in Fraction
        B = Fraction(param)
        C = (1 - B) / 2
        if t < 1:
            return ((12 - 9 * B - 6 * C) * t ** 3 + (-18 + 12 * B + 6 * C) * t ** 2 + (6 - 2 * B)) / 6
        if t < 2:
            return ((-B - 6 * C) * t ** 3 + (6 * B + 30 * C) * t ** 2 + (-12 * B - 48 * C) * t + (8 * B + 24 * C)) / 6
        return Fraction(0)
    if kernel == "gaussian":
        s = float(param)
        if t >= math.ceil(3 * s):
            return 0.0
        return math.exp(-float(x) ** 2 / (2 * s * s))
    if kernel == "lanczos":
        R = int(param)
        if t >= R:
            return 0.0
        if x == 0:
            return 1.0
        xf = float(x)
        return (math.sin(math.pi * xf) / (math.pi * xf)) * (
            math.sin(math.pi * xf / R) / (math.pi * xf / R))
    raise ValueError(kernel)


def scale_factor(n_in: int, n_out: int, antialias: bool = True) -> Fraction:
    if antialias and n_in > n_out:
        return Fraction(n_in, n_out)
    return Fraction(1)


@functools.lru_cache(maxsize=None)
def tap_set(n_in: int, n_out: int, i: int, R: int, antialias: bool = True):
    """Every integer j with |j + 1/2 - c_i| / sc < R, by exhaustive scan."""
    c = (i + Fraction(1, 2)) * Fraction(n_in, n_out)
    sc = scale_factor(n_in, n_out, antialias)
    lo = -(R + 2) * (n_in + n_out) - 8
    hi = (R + 2) * (n_in + n_out) + 8
    return tuple(j for j in range(lo, hi + 1) if abs(j + Fraction(1, 2) - c) / sc < R)


def map_index(j: int, n: int, boundary: str):
    """Boundary map by walking the extended signal one step at a time."""
    if boundary == "truncate":
        return j if 0 <= j < n else None
    if boundary == "clamp":
        return min(max(j, 0), n - 1)
    if boundary in ("mirror", "reflect101"):
        # unfold the symmetric extension explicitly: build one period
        if boundary == "mirror":
            period = list(range(n)) + list(range(n - 1, -1, -1))
        else:
            period = list(range(n)) + list(range(n - 2, 0, -1)) if n > 1 else [0]
        return period[j % len(period)]
    raise ValueError(boundary)


def axis_matrix(n_in: int, n_out: int, kernel: str, boundary: str, param=None,
                antialias: bool = True):
    """Dense n_out x n_in matrix (list of lists) of one axis."""
    if param is None:
        param = {"linear": 0, "cubic": Fraction(-1, 2), "lanczos": 3, "bspline3": 0, "mitchell": Fraction(1, 3),
                 "gaussian": 0.5}[kernel]
    R = support(kernel, param)
    sc = scale_factor(n_in, n_out, antialias)
    M = []
    for i in range(n_out):
        c = (i + Fraction(1, 2)) * Fraction(n_in, n_out)
        row = [Fraction(0)] * n_in if kernel not in ("lanczos", "gaussian") else [0.0] * n_in
        taps = tap_set(n_in, n_out, i, R, antialias)
        ws, ms = [], []
        for j in taps:
            m = map_index(j, n_in, boundary)
            if m is None:
                continue
            ws.append(kernel_exact(kernel, (j + Fraction(1, 2) - c) / sc, param))
            ms.append(m)
        s = sum(ws)
        for m, w in zip(ms, ws):
            row[m] += w / s
        M.append(row)
    return M


def resample(img, out_h: int, out_w: int, kernel: str, boundary: str, param=None,
             antialias: bool = True):
    """img: nested list [H][W][C] (numbers).  Returns nested list of floats."""
    H, W, C = len(img), len(img[0]), len(img[0][0])
    Mh = axis_matrix(H, out_h, kernel, boundary, param, antialias)
    Mw = axis_matrix(W, out_w, kernel, boundary, param, antialias)
    out = []
    for y in range(out_h):
        row = []
        for x in range(out_w):
            px = []
            for c in range(C):
                acc = 0
                for j in range(H):
                    if Mh[y][j] == 0:
                        continue
                    inner = 0
                    for i in range(W):
                        if Mw[x][i] != 0:
                            inner += Mw[x][i] * img[j][i][c]
                    acc += Mh[y][j] * inner
                px.append(float(acc))
            row.append(px)
        out.append(row)
    return out
