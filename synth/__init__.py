"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds no resampling arithmetic (not even the output-size rule):
it only draws pixels, image sizes, scales, kernels and request arrival times with numpy's PCG64
generator, so that the CUDA path and the CPU oracle are fed identical data.

Workloads (the paper this project accompanies measures nothing of this kind,
so each recipe is stated here and in the design notes):
  * uniform:   i.i.d. U[0, 1) pixels;
  * sinusoids: per channel, 0.5 + (0.25 / sqrt(32)) * sum of 64 plane waves
               sin(2 pi (f cos(theta) x + f sin(theta) y) + phi) with
               f ~ U[0, 0.45] cycles/pixel, theta ~ U[0, pi), phi ~ U[0, 2 pi),
               plus N(0, 0.05^2) noise, clipped to [0, 1];
  * batch:     512 single-channel images, H and W ~ U{64..2048} drawn
               independently, scale ~ logU[1/4, 4] (one per image, both axes),
               kernel ~ U{linear, cubic a=-1/2, Lanczos-3};
  * serving:   Poisson arrivals at 2000 req/s for 60 s, square images with
               side ~ logU[32, 4096], channels 1 or 3 (p = 1/2),
               scale ~ logU[1/8, 8], kernel ~ U{cubic a=-1/2, Lanczos-3};
  * ToF frames (the clustering workload): 204 x 204 depth / distance /
               intensity frames of a piecewise-planar scene -- a tilted
               background plane at 1.5-3 m and 3-6 tilted rectangles at
               0.5-1.5 m, each surface with a reflectivity in [0.2, 1];
               pinhole camera (focal length 200 px, centre at the middle):
               radial distance d = z sqrt(1 + r^2 / f^2), intensity
               I = reflectivity / d^2; noise N(0, 3 mm) on z (d follows it)
               and 1% multiplicative noise on I.  float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_C1 = 11105450
SEED_C2 = 11105451
SEED_C4 = 11105452
SEED_C5 = 11105453
SEED_TOF = 11105454


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(h: int, w: int, c: int = 1, seed: int = SEED_C1) -> np.ndarray:
    """(h, w, c) float64 i.i.d. U[0, 1)."""
    return rng(seed).random((h, w, c))


def sinusoids(h: int, w: int, c: int = 3, seed: int = SEED_C2, n_waves: int = 64,
              noise: float = 0.05) -> np.ndarray:
    """(h, w, c) float32 sum-of-plane-waves content plus noise, clipped to [0, 1].

    Each wave sin(a x + b y + phi) is expanded as
    sin(a x + phi) cos(b y) + cos(a x + phi) sin(b y), so a channel is one
    (h x 2K) @ (2K x w) product instead of h*w*K sine evaluations.
    """
    g = rng(seed)
    x = np.arange(w, dtype=np.float64)
    y = np.arange(h, dtype=np.float64)
    out = np.empty((h, w, c), dtype=np.float32)
    amp = 0.25 / math.sqrt(n_waves / 2.0)
    for ch in range(c):
        f = g.uniform(0.0, 0.45, n_waves)
        th = g.uniform(0.0, math.pi, n_waves)
        ph = g.uniform(0.0, 2.0 * math.pi, n_waves)
        a = 2.0 * math.pi * f * np.cos(th)
        b = 2.0 * math.pi * f * np.sin(th)
        ax = a[:, None] * x[None, :] + ph[:, None]          # (K, w)
        by = y[:, None] * b[None, :]                          # (h, K)
        left = np.concatenate([np.cos(by), np.sin(by)], axis=1)       # (h, 2K)
        right = np.concatenate([np.sin(ax), np.cos(ax)], axis=0)      # (2K, w)
        img = 0.5 + amp * (left @ right)
        img += g.normal(0.0, noise, (h, w))
        np.clip(img, 0.0, 1.0, out=img)
        out[:, :, ch] = img
    return out


@dataclass
class ImageSpec:
    in_h: int
    in_w: int
    channels: int
    scale: float
    kernel: str
    param: float
    seed: int


def batch_specs(n: int = 512, seed: int = SEED_C4, side=(64, 2048), scale=(0.25, 4.0)):
    """The uneven batch: one ImageSpec per image (single channel)."""
    g = rng(seed)
    kernels = [("linear", 0.0), ("cubic", -0.5), ("lanczos", 3.0)]
    specs = []
    for i in range(n):
        h = int(g.integers(side[0], side[1] + 1))
        w = int(g.integers(side[0], side[1] + 1))
        s = float(math.exp(g.uniform(math.log(scale[0]), math.log(scale[1]))))
        k, p = kernels[int(g.integers(0, 3))]
        specs.append(ImageSpec(h, w, 1, s, k, p, seed * 1000 + i))
    return specs


@dataclass
class Request:
    arrival_s: float
    spec: ImageSpec


def serving_trace(rate: float = 2000.0, duration_s: float = 60.0, seed: int = SEED_C5,
                  side=(32, 4096), scale=(0.125, 8.0)):
    """Open-loop Poisson arrivals; each request a square image spec."""
    g = rng(seed)
    kernels = [("cubic", -0.5), ("lanczos", 3.0)]
    t = 0.0
    reqs = []
    i = 0
    while True:
        t += float(g.exponential(1.0 / rate))
        if t >= duration_s:
            break
        n = int(round(math.exp(g.uniform(math.log(side[0]), math.log(side[1])))))
        c = 1 if g.random() < 0.5 else 3
        s = float(math.exp(g.uniform(math.log(scale[0]), math.log(scale[1]))))
        k, p = kernels[int(g.integers(0, 2))]
        reqs.append(Request(t, ImageSpec(n, n, c, s, k, p, seed * 1000 + i)))
        i += 1
    return reqs


def tof_frames(n: int, h: int = 204, w: int = 204, seed: int = SEED_TOF):
    """(z, d, intensity): three (n, h, w) float32 arrays of synthetic ToF frames."""
    g = rng(seed)
    v, u = np.mgrid[0:h, 0:w].astype(np.float64)
    f_px, cx, cy = 200.0, (w - 1) / 2.0, (h - 1) / 2.0
    ray = np.sqrt(1.0 + ((u - cx) ** 2 + (v - cy) ** 2) / f_px ** 2)
    Z = np.empty((n, h, w), np.float32)
    D = np.empty((n, h, w), np.float32)
    I = np.empty((n, h, w), np.float32)
    for k in range(n):
        z = g.uniform(1.5, 3.0) + g.uniform(-0.002, 0.002) * (u - cx) + g.uniform(-0.002, 0.002) * (v - cy)
        refl = np.full((h, w), g.uniform(0.2, 1.0))
        for _ in range(int(g.integers(3, 7))):
            y0, x0 = int(g.integers(0, h - 8)), int(g.integers(0, w - 8))
            y1, x1 = int(g.integers(y0 + 8, min(h, y0 + h // 2) + 1)), int(g.integers(x0 + 8, min(w, x0 + w // 2) + 1))
            zc = g.uniform(0.5, 1.5)
            gy, gx = g.uniform(-0.003, 0.003), g.uniform(-0.003, 0.003)
            sl = (slice(y0, y1), slice(x0, x1))
            z[sl] = zc + gx * (u[sl] - x0) + gy * (v[sl] - y0)
            refl[sl] = g.uniform(0.2, 1.0)
        z = z + g.normal(0.0, 0.003, (h, w))
        d = z * ray
        inten = refl / (d * d) * (1.0 + g.normal(0.0, 0.01, (h, w)))
        Z[k], D[k], I[k] = z, d, np.maximum(inten, 1e-6)
    return Z, D, I
