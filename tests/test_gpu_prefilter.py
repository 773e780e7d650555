"""Interpolating cubic B-spline (RS_PREFILTER) against the FP64 oracle.

The device replaces the input by its B-spline coefficients (one tridiagonal
solve per row, then per column) and resamples them with the cubic B-spline on
whichever kernel path the plan takes; the oracle solves the same
interpolation condition as a dense linear system.  FP32 (2e-6) and FP64
(1e-12), 1 and 3 channels, the clamp / mirror / reflect101 boundaries,
identity, up- and downscales, every kernel path that applies.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TOL, quantise, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_5450_b300 as rs

    return rs


SHAPES = [((37, 44), (37, 44)),     # identity: the samples come back
          ((40, 52), (91, 117)),    # x2.27 up
          ((96, 132), (131, 181)),  # ~x1.37
          ((120, 88), (36, 27)),    # ~x0.3 down
          ((1, 9), (3, 20)),        # one row
          ((2, 2), (5, 5))]         # two samples per axis
PATHS = {"default": 0, "tile": "SIMT|NO_STREAM", "stream": "FORCE_STREAM", "vfirst": "FORCE_VFIRST",
         "two_pass": "TWO_PASS"}


def _flags(rs, spec):
    if spec == 0:
        return 0
    f = 0
    for name in spec.split("|"):
        f |= getattr(rs, "RS_" + ("FORCE_SIMT" if name == "SIMT" else name))
    return f


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a[0]}x{a[1]}-{b[0]}x{b[1]}" for a, b in SHAPES])
@pytest.mark.parametrize("boundary", ["clamp", "mirror", "reflect101"])
@pytest.mark.parametrize("C", [1, 3])
def test_prefilter_parity(rs, dt, path, shape, boundary, C):
    (H, W), (OH, OW) = shape
    flags = rs.RS_PREFILTER | _flags(rs, PATHS[path])
    img = synth.uniform(H, W, C, seed=(H * 3 + W + C) & 0xffff)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, OH, OW, "bspline3", boundary, prefilter=True)
    try:
        got, info = run_gpu(t, OH, OW, "bspline3", boundary, None, flags)
    except RuntimeError as e:
        # forced kernels that do not take this plan (FP64, an upscale in rows
        # for the vertical-first kernels, rows narrower than a TMA word)
        assert "unsupported" in str(e) and path in ("stream", "vfirst", "tile"), e
        return
    err = np.abs(got - want).max()
    assert err <= TOL[dt], (err, info.path)
    if (H, W) == (OH, OW):
        assert np.abs(got - exact).max() <= TOL[dt]


def test_prefilter_full_size_sampled_rows(rs):
    """4096x4096x3 FP32 x1.37 on the default (streaming) plan, sampled rows."""
    t, exact = quantise(synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2), "f32")
    got, info = run_gpu(t, 0, 0, "bspline3", "mirror", None, rs.RS_PREFILTER, scale=1.37)
    coef = oracle.bspline_coefficients(exact, "mirror")
    g = np.random.default_rng(2)
    rows = sorted(set([0, 2805, 5611]) | set(int(r) for r in g.integers(0, 5612, 5)))
    err = 0.0
    for r in rows:
        want = oracle.resample(coef, 5612, 5612, "bspline3", "mirror", rows=(r, r + 1))
        err = max(err, float(np.abs(got[r] - want[0]).max()))
    assert err <= TOL["f32"], err


def test_prefilter_not_in_batches(rs):
    import torch

    with pytest.raises(RuntimeError, match="unsupported"):
        rs.Batch([dict(in_h=32, in_w=32, scale=2.0, kernel="bspline3", boundary="mirror",
                       flags=rs.RS_PREFILTER)], channels=1, dtype=torch.float32)
