"""Mitchell-Netravali and Gaussian kernels on every kernel path, against the
FP64 oracle: the default plan, the tile kernel, the row-streaming kernel, the
vertical-first and the plain two-pass kernels, and (16-bit) the tensor-core
tiles; upscales and antialiased downscales, 1 and 3 channels, every boundary.
Tolerances FP32 2e-6, BF16 1e-2 (max-abs on [0, 1] data)."""
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


SHAPES = [((64, 96), (150, 203)),   # x2.2 up
          ((200, 168), (60, 50))]   # ~x0.3 down (antialiased)
PATHS = ["default", "tile", "stream", "vfirst", "two_pass", "tcgen05"]


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("shape", SHAPES, ids=["up", "down"])
@pytest.mark.parametrize("kernel,param", [("mitchell", 1.0 / 3.0), ("mitchell", 0.0), ("gaussian", 0.5),
                                          ("gaussian", 1.0)])
@pytest.mark.parametrize("boundary", ["clamp", "mirror", "reflect101", "truncate"])
@pytest.mark.parametrize("C", [1, 3])
def test_new_kernels(rs, dt, path, shape, kernel, param, boundary, C):
    (H, W), (OH, OW) = shape
    flags = {"default": 0, "tile": rs.RS_FORCE_SIMT | rs.RS_NO_STREAM, "stream": rs.RS_FORCE_STREAM,
             "vfirst": rs.RS_FORCE_VFIRST, "two_pass": rs.RS_TWO_PASS, "tcgen05": rs.RS_FORCE_TC}[path]
    if path == "tcgen05" and dt == "f32":
        pytest.skip("tensor-core tiles take 16-bit storage only")
    if path == "vfirst" and OH > H:
        pytest.skip("vertical-first needs out_h <= in_h")
    img = synth.uniform(H, W, C, seed=(H + 3 * W + 7 * C) & 0xffff)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
    got, info = run_gpu(t, OH, OW, kernel, boundary, param, flags)
    expect = {"tile": 0, "stream": 3, "vfirst": 4, "two_pass": 1, "tcgen05": 2}.get(path)
    if path == "stream" and dt != "f32" and OH < H:
        # a forced streaming 16-bit downscale with wide windows runs stream form 3 (plan path 5)
        assert info.path in (3, 5)
    elif expect is not None:
        assert info.path == expect
    assert np.abs(got - want).max() <= TOL[dt], (np.abs(got - want).max(), info.path)


def test_kernel_parameter_range(rs):
    import torch

    for kernel, param in (("mitchell", -0.1), ("mitchell", 1.5), ("gaussian", 0.0), ("gaussian", 4.5)):
        with pytest.raises(RuntimeError):
            rs.Plan(32, 32, 1, 16, 16, kernel=kernel, param=param, boundary="mirror", dtype=torch.float32)
