"""Checks that pin the FP64 oracle to facts outside itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` instance and raises
AssertionError when that instance disagrees with a closed form, a published
kernel value, a library routine (numpy.pad, torch.nn.functional.interpolate in
float64 on the CPU), an exact-rational brute force, or an invariant of the
mathematics.  ``test_oracle_pins.py`` runs them on the real oracle and
``test_oracle_mutants.py`` runs them on deliberately broken copies, each of
which must fail at least one pin.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

from oracle import brute

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
KERNELS = ["linear", "cubic", "lanczos", "bspline3", "mitchell", "gaussian"]
BOUNDARIES = ["clamp", "mirror", "reflect101", "truncate"]


def _rng(seed):
    return np.random.default_rng(seed)


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _parse_value(tok):
    if tok.endswith("/pi2"):
        p, q, _ = tok.split("/")
        return float(Fraction(int(p), int(q))) / (math.pi ** 2)
    p, q = tok.split("/")
    return float(Fraction(int(p), int(q)))


# ---------------------------------------------------------------- closed forms
def pin_kernel_values(o):
    """Published kernel definitions at points with closed-form values."""
    for kernel, param, x, val in _read_rows("kernel_values.txt"):
        got = o.kernel_value(kernel, float(x), float(param))
        want = _parse_value(val)
        assert abs(got - want) <= 4e-16 * max(1.0, abs(want)), (kernel, param, x, got, want)


def pin_keys_x2(o):
    """Keys a=-1/2 at exact x2 upscaling: dyadic weights, bit-exact."""
    want = {r[0]: [Fraction(int(v), 128) for v in r[1:]] for r in _read_rows("keys_cubic_x2_weights.txt")}
    rows = o.axis_weights(256, 512, "cubic", "clamp", param=-0.5)
    for i in range(4, 508):
        jf, idx, w = rows[i]
        parity = "even" if i % 2 == 0 else "odd"
        assert len(w) == 4, (i, len(w))
        assert [Fraction(float(v)) for v in w] == want[parity], (i, w)
        assert list(idx) == list(range(jf, jf + 4))


def pin_bilinear_aa_half(o):
    """Tent filter widened by 2 at exact 1/2 downscaling: {1,3,3,1}/8."""
    want = [Fraction(int(v), 8) for v in _read_rows("bilinear_aa_half_weights.txt")[0]]
    rows = o.axis_weights(64, 32, "linear", "clamp")
    for i in range(2, 30):
        jf, idx, w = rows[i]
        assert [Fraction(float(v)) for v in w] == want, (i, w)
        assert jf == 2 * i - 1


def pin_identity(o):
    """n_in == n_out: interpolating kernels reproduce the samples exactly;
    the cubic B-spline (approximating) applies the [1, 4, 1] / 6 smoother."""
    img = _rng(1).random((13, 17, 2))
    for kernel in ("linear", "cubic", "lanczos"):
        for boundary in BOUNDARIES:
            out = o.resample(img, 13, 17, kernel, boundary)
            assert np.array_equal(out, img), (kernel, boundary, np.abs(out - img).max())
    out = o.resample(img, 13, 17, "bspline3", "mirror")
    pad = np.pad(img, ((1, 1), (1, 1), (0, 0)), mode="symmetric")
    s = (pad[:-2] + 4 * pad[1:-1] + pad[2:]) / 6
    s = (s[:, :-2] + 4 * s[:, 1:-1] + s[:, 2:]) / 6
    assert np.abs(out - s).max() < 1e-15


def pin_constant(o):
    """Partition of unity after normalisation: a constant image stays constant."""
    img = np.full((11, 7, 3), 0.37)
    for kernel in KERNELS:
        for boundary in BOUNDARIES:
            for oh, ow in ((11, 7), (23, 3), (4, 15), (1, 1), (2, 29)):
                out = o.resample(img, oh, ow, kernel, boundary)
                assert np.abs(out - 0.37).max() < 1e-14, (kernel, boundary, oh, ow)


def _moments(rows, n_in, n_out, lo, hi):
    """Discrete moments sum_k w_k d_k^p at outputs [lo, hi), d = j + 1/2 - c_i."""
    res = []
    for i in range(lo, hi):
        jf, idx, w = rows[i]
        j = np.arange(jf, jf + len(w))
        d = (j + 0.5) - (i + 0.5) * n_in / n_out
        res.append([float(np.sum(w * d ** p)) for p in range(4)])
    return np.array(res)


def pin_polynomials(o):
    """Polynomial reproduction at scale >= 1, interior outputs:
    Keys a=-1/2 reproduces degree <= 2, the tent degree <= 1, the cubic B-spline
    has second moment exactly 1/3 (x^2 -> x^2 + 1/3), Keys a=-3/4 does not
    reproduce linear functions and Lanczos-3 only constants."""
    for n_in, n_out in ((16, 37), (20, 20), (12, 29), (9, 64)):
        lo, hi = 3 * n_out // n_in + 3, n_out - 3 * n_out // n_in - 3
        m = _moments(o.axis_weights(n_in, n_out, "cubic", "clamp", param=-0.5), n_in, n_out, lo, hi)
        assert np.abs(m[:, 0] - 1).max() < 1e-14 and np.abs(m[:, 1]).max() < 1e-13
        assert np.abs(m[:, 2]).max() < 1e-13
        m = _moments(o.axis_weights(n_in, n_out, "linear", "clamp"), n_in, n_out, lo, hi)
        assert np.abs(m[:, 1]).max() < 1e-14
        m = _moments(o.axis_weights(n_in, n_out, "bspline3", "clamp"), n_in, n_out, lo, hi)
        assert np.abs(m[:, 1]).max() < 1e-14 and np.abs(m[:, 2] - 1 / 3).max() < 1e-14
        assert np.abs(m[:, 3]).max() < 1e-13
    m = _moments(o.axis_weights(16, 37, "cubic", "clamp", param=-0.75), 16, 37, 6, 31)
    assert np.abs(m[:, 1]).max() > 0.01
    m = _moments(o.axis_weights(16, 37, "lanczos", "clamp"), 16, 37, 8, 29)
    assert np.abs(m[:, 1]).max() > 1e-4


def pin_polynomial_image(o):
    """2-D: Keys a=-1/2 upscaling of a quadratic surface p(u, v) sampled at
    input centres reproduces p at the output centres (interior).  The surface
    is asymmetric in u and v and the grid is not square, so an axis or index
    mix-up fails here."""
    H, W, OH, OW = 10, 14, 23, 31

    def p(u, v):
        return 0.3 + 0.02 * u - 0.015 * v + 0.003 * u * u + 0.001 * u * v - 0.002 * v * v

    u = np.arange(H)[:, None] + 0.5
    v = np.arange(W)[None, :] + 0.5
    img = np.stack([p(u, v), 2 * p(u, v)], axis=-1)
    out = o.resample(img, OH, OW, "cubic", "clamp", param=-0.5)
    uo = (np.arange(OH)[:, None] + 0.5) * H / OH
    vo = (np.arange(OW)[None, :] + 0.5) * W / OW
    want = p(uo, vo)
    sl = (slice(5, OH - 5), slice(5, OW - 5))
    assert np.abs(out[..., 0][sl] - want[sl]).max() < 1e-13
    assert np.abs(out[..., 1][sl] - 2 * want[sl]).max() < 2e-13


# ----------------------------------------------------------- library cross-check
def pin_torch(o):
    """torch.nn.functional.interpolate (CPU, float64, align_corners=False):
    bicubic = Keys a=-3/4 + clamp; bilinear = tent + clamp; with antialias=True
    the kernel is widened by the scale and out-of-range taps are dropped and
    the rest renormalised (truncate), with a=-1/2 for bicubic."""
    import torch
    import torch.nn.functional as F

    img = _rng(2).random((9, 11, 3))
    t = torch.from_numpy(img).permute(2, 0, 1)[None]
    cases = [
        ((13, 17), "bicubic", False, "cubic", -0.75, "clamp", False),
        ((5, 7), "bicubic", False, "cubic", -0.75, "clamp", False),
        ((13, 17), "bilinear", False, "linear", 0.0, "clamp", False),
        ((4, 6), "bilinear", False, "linear", 0.0, "clamp", False),
        ((4, 5), "bilinear", True, "linear", 0.0, "truncate", True),
        ((4, 5), "bicubic", True, "cubic", -0.5, "truncate", True),
        ((3, 2), "bicubic", True, "cubic", -0.5, "truncate", True),
        ((20, 23), "bicubic", True, "cubic", -0.5, "truncate", True),
    ]
    for size, mode, aa, kernel, param, boundary, ours_aa in cases:
        ref = F.interpolate(t, size=size, mode=mode, align_corners=False, antialias=aa)
        ref = ref[0].permute(1, 2, 0).numpy()
        out = o.resample(img, size[0], size[1], kernel, boundary, param=param, antialias=ours_aa)
        assert np.abs(out - ref).max() < 1e-14, (size, mode, aa, np.abs(out - ref).max())


def pin_boundary_pad(o):
    """Boundary maps against numpy.pad: 'edge' = clamp, 'symmetric' = mirror
    (half-sample symmetric), 'reflect' = reflect101; far taps fold repeatedly."""
    for n in range(1, 10):
        P = 4 * n + 5
        base = np.arange(n)
        for mode, b in (("edge", "clamp"), ("symmetric", "mirror"), ("reflect", "reflect101")):
            padded = np.pad(base, P, mode=mode)
            for j in range(-P, n + P):
                assert o.boundary_map(j, n, b) == padded[j + P], (n, mode, j)
        for j in range(-P, n + P):
            assert o.boundary_map(j, n, "truncate") == (j if 0 <= j < n else -1)


# ------------------------------------------------------------ exact brute force
def pin_taps_fractions(o):
    """Integer tap test against an exact-rational scan of the definition, all
    (n_in, n_out) in 1..16, with and without antialiasing."""
    for kernel, R in (("linear", 1), ("cubic", 2), ("lanczos", 3)):
        for aa in (True, False):
            for n_in in range(1, 17):
                for n_out in range(1, 17):
                    for i in range(n_out):
                        js = brute.tap_set(n_in, n_out, i, R, aa)
                        jf, cnt = o.axis_taps(n_in, n_out, kernel, i, antialias=aa)
                        assert (jf, cnt) == (js[0], len(js)), (kernel, aa, n_in, n_out, i)


def pin_brute(o):
    """Whole resampling against the dense-matrix brute force on tiny grids."""
    rng = _rng(3)
    shapes = [((1, 1), (3, 2)), ((2, 3), (5, 1)), ((5, 3), (2, 7)), ((4, 6), (4, 6)), ((7, 2), (3, 3))]
    for (H, W), (OH, OW) in shapes:
        img = rng.random((H, W, 2))
        for kernel in KERNELS:
            for boundary in BOUNDARIES:
                want = np.array(brute.resample(img.tolist(), OH, OW, kernel, boundary))
                got = o.resample(img, OH, OW, kernel, boundary)
                assert np.abs(got - want).max() < 1e-13, (H, W, OH, OW, kernel, boundary)


# ------------------------------------------------ Mitchell-Netravali, Gaussian
def pin_mitchell_gaussian(o):
    """Mitchell-Netravali on the B + 2C = 1 line: B = 0 is Keys a = -1/2, B = 1
    the cubic B-spline; for every B the integer shifts sum to 1, the first
    moment vanishes and the second is B / 3 (D. Mitchell, A. Netravali,
    SIGGRAPH 1988).  Gaussian: exp(-x^2 / 2 sigma^2) at sigma and 2 sigma,
    zero from the truncation radius ceil(3 sigma) on."""
    xs = np.linspace(-2.5, 2.5, 201)
    for x in xs:  # the same polynomials in other forms: a few ulps of the coefficients (~24)
        assert abs(o.kernel_value("mitchell", x, 0.0) - o.kernel_value("cubic", x, -0.5)) < 1e-14
        assert abs(o.kernel_value("mitchell", x, 1.0) - o.kernel_value("bspline3", x)) < 1e-14
    for B in (0.0, 1 / 3, 0.5, 0.8, 1.0):
        for x in np.linspace(0.0, 0.99, 34):
            ks = [(x + k, o.kernel_value("mitchell", x + k, B)) for k in range(-3, 4)]
            assert abs(sum(w for _, w in ks) - 1.0) < 1e-14, (B, x)
            assert abs(sum(d * w for d, w in ks)) < 1e-14, (B, x)
            assert abs(sum(d * d * w for d, w in ks) - B / 3) < 1e-14, (B, x)
    for s in (0.5, 0.8, 1.3):
        R = math.ceil(3 * s)
        assert o.kernel_value("gaussian", 0.0, s) == 1.0
        assert abs(o.kernel_value("gaussian", s, s) - math.exp(-0.5)) < 1e-16
        assert abs(o.kernel_value("gaussian", -2 * s, s) - math.exp(-2.0)) < 1e-16
        assert o.kernel_value("gaussian", R, s) == 0.0 and o.kernel_value("gaussian", -R, s) == 0.0
        assert o.kernel_value("gaussian", R - 1e-9, s) > 0.0


# ---------------------------------------------- interpolating cubic B-spline
def pin_prefilter(o):
    """B-spline coefficients from the interpolation condition: the prefiltered
    B-spline reproduces the samples at scale 1 (every boundary rule); the
    coefficients equal scipy's recursive spline filter (its 'reflect' is the
    half-sample 'mirror' here, its 'mirror' the whole-sample 'reflect101'),
    and resampling equals scipy's cubic spline interpolation at the same
    half-pixel coordinates."""
    import scipy.ndimage as nd

    rng = _rng(5)
    img = rng.random((13, 11, 2))
    for boundary in ("clamp", "mirror", "reflect101"):
        out = o.resample(img, 13, 11, "bspline3", boundary, prefilter=True)
        assert np.abs(out - img).max() < 1e-13, boundary
    for boundary, mode in (("mirror", "reflect"), ("reflect101", "mirror")):
        for n in (1, 2, 3, 9, 40):
            x = rng.random(n)
            c = o.bspline_coefficients(x[:, None], boundary)[:, 0]
            assert np.abs(c - nd.spline_filter1d(x, order=3, mode=mode)).max() < 1e-13, (boundary, n)
        src = rng.random((20, 24))
        for oh, ow in ((40, 48), (31, 37), (20, 24)):
            out = o.resample(src, oh, ow, "bspline3", boundary, prefilter=True)
            yy = (np.arange(oh) + 0.5) * 20 / oh - 0.5
            xx = (np.arange(ow) + 0.5) * 24 / ow - 0.5
            Y, X = np.meshgrid(yy, xx, indexing="ij")
            ref = nd.map_coordinates(src, [Y, X], order=3, mode=mode, prefilter=True)
            assert np.abs(out - ref).max() < 1e-13, (boundary, oh, ow)


# --------------------------------------------------------------------- invariants
def pin_invariants(o):
    """Linearity, transpose symmetry and channel independence."""
    rng = _rng(4)
    X = rng.random((12, 12, 3))
    Y = rng.random((12, 12, 3))
    for kernel in KERNELS:
        rx = o.resample(X, 17, 17, kernel, "mirror")
        ry = o.resample(Y, 17, 17, kernel, "mirror")
        rxy = o.resample(0.25 * X - 1.5 * Y, 17, 17, kernel, "mirror")
        assert np.abs(rxy - (0.25 * rx - 1.5 * ry)).max() < 1e-13
        rt = o.resample(X.transpose(1, 0, 2), 17, 17, kernel, "mirror")
        assert np.abs(rt - rx.transpose(1, 0, 2)).max() < 1e-14
        for c in range(3):
            rc = o.resample(X[:, :, c], 17, 17, kernel, "mirror")
            assert np.array_equal(rc, rx[:, :, c])


ALL_PINS = [pin_kernel_values, pin_keys_x2, pin_bilinear_aa_half, pin_identity, pin_constant,
            pin_polynomials, pin_polynomial_image, pin_torch, pin_boundary_pad,
            pin_taps_fractions, pin_brute, pin_invariants, pin_mitchell_gaussian, pin_prefilter]
