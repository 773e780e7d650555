"""Affine EWA warps on the GPU against the FP64 oracle: identity, scalings up
and down, rotations, shears, anisotropic and translated maps, every boundary,
1 and 3 channels, FP32 / FP16 / BF16 storage, strided buffers.

Tolerance: the resampler's, FP32 2e-6 max-abs on [0, 1] data (measured
2.5e-7 to 5e-7: the kernel forms its FP32 weights exp(-Q/2) from offsets
exact to FP32 rounding and normalises by their FP32 sum), FP16 2e-3, BF16
1e-2 (the storage rounding).  The oracle is fed the same quantised input."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import TOL, quantise
from oracle import warp as ow

pytestmark = pytest.mark.gpu

TOLW = {"f32": TOL["f32"], "f16": TOL["f16"], "bf16": TOL["bf16"]}


@pytest.fixture(scope="module")
def rs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_5450_b300 as rs

    return rs


def _rot(deg, s, cx, cy, ox, oy):
    """Output centre (ox, oy) maps to input centre (cx, cy), rotated by deg and scaled by s (input per output)."""
    c, n = math.cos(math.radians(deg)) * s, math.sin(math.radians(deg)) * s
    return (c, -n, cx - c * ox + n * oy, n, c, cy - n * ox - c * oy)


MAPS = {
    "identity": ((40, 48), (40, 48), (1, 0, 0, 0, 1, 0)),
    "down3": ((60, 72), (20, 24), (3, 0, 0, 0, 3, 0)),
    "up2.5": ((16, 20), (40, 50), (0.4, 0, 0, 0, 0.4, 0)),
    "rot30": ((40, 40), (36, 36), _rot(30, 1.0, 20, 20, 18, 18)),
    "rot75_down": ((64, 64), (24, 24), _rot(75, 2.2, 32, 32, 12, 12)),
    "shear": ((36, 44), (30, 40), (1.0, 0.45, -4.0, 0.1, 1.2, 1.5)),
    "aniso": ((50, 60), (40, 15), (4.0, 0.0, 0.0, 0.0, 1.25, 0.0)),
    "outside": ((20, 24), (16, 16), (1.0, 0.0, 15.0, 0.0, 1.0, -6.0)),
}


@pytest.mark.parametrize("name", list(MAPS))
@pytest.mark.parametrize("boundary", ["clamp", "mirror", "reflect101", "truncate"])
@pytest.mark.parametrize("C", [1, 3])
def test_warp_parity_fp32(rs, name, boundary, C):
    import torch

    (H, W), (OH, OW), a = MAPS[name]
    img = synth.uniform(H, W, C, seed=H + 7 * W + C)
    x = torch.from_numpy(img.astype(np.float32)).cuda()
    y = rs.warp(x, OH, OW, a, sigma=0.5, cutoff=3.0, boundary=boundary)
    torch.cuda.synchronize()
    want = ow.warp(img.astype(np.float32).astype(np.float64), OH, OW, a, 0.5, 3.0, boundary)
    assert np.abs(y.double().cpu().numpy() - want).max() <= TOLW["f32"]


@pytest.mark.parametrize("dt", ["f16", "bf16"])
@pytest.mark.parametrize("name", ["rot30", "down3", "up2.5"])
def test_warp_parity_16bit(rs, dt, name):
    import torch

    (H, W), (OH, OW), a = MAPS[name]
    t, exact = quantise(synth.uniform(H, W, 3, seed=5), dt)
    y = rs.warp(t.cuda(), OH, OW, a, sigma=0.7, cutoff=2.5, boundary="mirror")
    torch.cuda.synchronize()
    want = ow.warp(exact, OH, OW, a, 0.7, 2.5, "mirror")
    assert np.abs(y.double().cpu().numpy() - want).max() <= TOLW[dt]


def test_warp_strided_buffers(rs):
    import torch

    H, W, C, OH, OW = 30, 34, 3, 25, 27
    a = _rot(20, 1.1, 17, 15, 13, 12)
    img = synth.uniform(H, W, C, seed=8).astype(np.float32)
    pin, pout = W * C + 7, OW * C + 5
    src = torch.zeros((H, pin), dtype=torch.float32, device="cuda")
    src[:, :W * C] = torch.from_numpy(img.reshape(H, W * C)).cuda()
    dst = torch.full((OH, pout), float("nan"), dtype=torch.float32, device="cuda")
    d = rs.rs_warp_desc(H, W, C, OH, OW, (rs.ctypes.c_double * 6)(*a), 0.5, 3.0, rs.RS_B_CLAMP, rs.RS_F32, pin, pout)
    rs.rs_warp(d, src.data_ptr(), dst.data_ptr(), 0)
    torch.cuda.synchronize()
    got = dst[:, :OW * C].double().cpu().numpy().reshape(OH, OW, C)
    want = ow.warp(img.astype(np.float64), OH, OW, a, 0.5, 3.0, "clamp")
    assert np.abs(got - want).max() <= TOLW["f32"]
    assert torch.isnan(dst[:, OW * C:]).all()


def test_warp_rejects_bad_descriptors(rs):
    import torch

    x = torch.zeros((8, 8, 1), device="cuda")
    for kw in (dict(sigma=0.0), dict(cutoff=9.0), dict(a=(float("nan"), 0, 0, 0, 1, 0))):
        args = dict(a=(1, 0, 0, 0, 1, 0), sigma=0.5, cutoff=3.0)
        args.update(kw)
        with pytest.raises(RuntimeError):
            rs.warp(x, 4, 4, **args)
