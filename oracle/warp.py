"""CPU oracle of the affine warp with elliptical weighted average (EWA)
filtering (TEST INFRASTRUCTURE ONLY; shares no code with the CUDA kernel).

Definition (P. Heckbert, "Fundamentals of Texture Mapping and Image
Warping", UC Berkeley 1989, ch. 3; N. Greene and P. Heckbert, IEEE CG&A 6(6),
1986), evaluated literally in FP64 per output pixel:

  * output pixel (x, y), centre p = (x + 1/2, y + 1/2), maps to the input point
    c = (a0 p_x + a1 p_y + a2, a3 p_x + a4 p_y + a5) (input sample (i, j) sits at
    (i + 1/2, j + 1/2));
  * the filter is the Gaussian reconstruction filter of standard deviation
    sigma (input pixels) convolved with the Gaussian prefilter of the same
    width in output pixels carried into the input by the Jacobian
    J = [[a0, a1], [a3, a4]]: covariance V = sigma^2 (J J^T + I);
  * input sample s contributes with Q = d^T V^-1 d, d = s - c, and weight
    exp(-Q / 2) - exp(-r^2 / 2) for Q < r^2 (r = `cutoff`), else 0 -- the
    Gaussian truncated at the ellipse Q = r^2 and lowered to reach zero
    there, so the weights are continuous (a reading: the sources truncate
    without saying how);
  * taps outside the image follow the boundary map (clamp, mirror,
    reflect101) or are dropped (truncate); out = sum w in / sum w (0 if no
    weight is left).
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def covariance(a, sigma):
    J = np.array([[a[0], a[1]], [a[3], a[4]]], dtype=np.float64)
    return (sigma * sigma) * (J @ J.T + np.eye(2))


def warp(img, out_h: int, out_w: int, a, sigma: float = 0.5, cutoff: float = 3.0, boundary: str = "clamp"):
    """img (H, W) or (H, W, C); a = (a0 .. a5); returns float64 (out_h, out_w[, C])."""
    src = np.asarray(img, dtype=np.float64)
    squeeze = src.ndim == 2
    if squeeze:
        src = src[:, :, None]
    H, W, C = src.shape
    V = covariance(a, sigma)
    Vi = np.linalg.inv(V)
    r2 = cutoff * cutoff
    wcut = math.exp(-r2 / 2.0)
    eu, ev = cutoff * math.sqrt(V[0, 0]), cutoff * math.sqrt(V[1, 1])
    mi = {i: oracle.boundary_map(i, W, boundary) for i in range(-W - 64, 2 * W + 64)}
    mj = {j: oracle.boundary_map(j, H, boundary) for j in range(-H - 64, 2 * H + 64)}
    out = np.zeros((out_h, out_w, C))
    for y in range(out_h):
        for x in range(out_w):
            cu = a[0] * (x + 0.5) + a[1] * (y + 0.5) + a[2]
            cv = a[3] * (x + 0.5) + a[4] * (y + 0.5) + a[5]
            i0, i1 = math.ceil(cu - eu - 0.5), math.floor(cu + eu - 0.5)
            j0, j1 = math.ceil(cv - ev - 0.5), math.floor(cv + ev - 0.5)
            acc, wsum = np.zeros(C), 0.0
            for j in range(j0, j1 + 1):
                dv = j + 0.5 - cv
                mj_ = mj.get(j, oracle.boundary_map(j, H, boundary))
                if mj_ < 0:
                    continue
                for i in range(i0, i1 + 1):
                    du = i + 0.5 - cu
                    q = Vi[0, 0] * du * du + 2.0 * Vi[0, 1] * du * dv + Vi[1, 1] * dv * dv
                    if q >= r2:
                        continue
                    mi_ = mi.get(i, oracle.boundary_map(i, W, boundary))
                    if mi_ < 0:
                        continue
                    w = math.exp(-q / 2.0) - wcut
                    acc += w * src[mj_, mi_]
                    wsum += w
            if wsum > 0.0:
                out[y, x] = acc / wsum
    return out[:, :, 0] if squeeze else out
