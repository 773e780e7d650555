"""The row-streaming kernel (plan path 3) against the FP64 oracle.

FP32 images of 1 and 3 channels, every kernel and boundary, upscales and mild
downscales with ragged strips and row ranges, forced onto the streaming kernel
and kept off it; the fallback to the tile kernel for an unaligned input; the
4096x4096x3 x1.37 configuration on sampled rows; recompute and autotune.
FP16 / BF16 storage (FP32 filtering, rounded stores) on the same cases where
rows are whole 16-byte words, and the 4096x4096x3 x1.37 / x0.3 cases on
sampled rows.  Tolerances FP32 2e-6, FP16 2e-3, BF16 1e-2 (max-abs on [0, 1]
data, the oracle fed the same quantised input).
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


SHAPES = [((67, 92), (150, 203)),     # x2.2, ragged strips
          ((96, 132), (131, 181)),    # ~x1.37
          ((300, 400), (411, 548)),   # x1.37, several row ranges
          ((33, 36), (33, 36)),       # identity
          ((64, 100), (50, 77)),      # mild downscale (~x0.78)
          ((40, 400), (90, 999)),     # wide, many strips
          ((200, 20), (401, 37)),     # tall, one strip
          ((32, 32), (5, 3)),         # tiny output
          ((300, 400), (90, 120)),    # x0.3: wide strips (two boxes per staged row)
          ((257, 611), (77, 183))]    # ~x0.3, ragged


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a[0]}x{a[1]}-{b[0]}x{b[1]}" for a, b in SHAPES])
@pytest.mark.parametrize("kernel,param", [("linear", None), ("cubic", -0.5), ("lanczos", 3.0),
                                          ("bspline3", None)])
@pytest.mark.parametrize("boundary", ["clamp", "mirror", "reflect101", "truncate"])
@pytest.mark.parametrize("C", [1, 3])
def test_stream_parity(rs, shape, kernel, param, boundary, C):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=(H * 31 + W * 7 + C) & 0xffff)
    t, exact = quantise(img, "f32")
    want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
    try:
        got, info = run_gpu(t, OH, OW, kernel, boundary, param, rs.RS_FORCE_STREAM)
    except RuntimeError as e:
        # only a band wider than the kernel takes (strong downscale) may refuse
        assert "unsupported" in str(e) and OH < H, e
        return
    assert info.path == 3
    err = np.abs(got - want).max()
    assert err <= TOL["f32"], (err, info.tile_w, info.span_h, info.span_w)
    tile, _ = run_gpu(t, OH, OW, kernel, boundary, param, rs.RS_NO_STREAM)
    assert np.abs(tile - want).max() <= TOL["f32"]


def test_stream_is_default_for_fp32_upscale(rs):
    import torch

    p = rs.Plan(4096, 4096, 3, scale=1.37, kernel="lanczos", param=3.0, boundary="mirror")
    assert p.path == "stream", p.path
    p.close()
    p = rs.Plan(4096, 4096, 3, scale=1.37, kernel="lanczos", param=3.0, boundary="mirror",
                flags=rs.RS_NO_STREAM)
    assert p.path == "fused"
    p.close()
    p = rs.Plan(4096, 4096, 3, scale=0.125, kernel="lanczos", param=3.0, boundary="mirror")
    assert p.path == "fused"   # band too wide for the streaming kernel
    p.close()
    with pytest.raises(RuntimeError, match="unsupported"):   # FP64 is not streamed
        rs.Plan(64, 64, 3, 100, 100, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float64,
                flags=rs.RS_FORCE_STREAM)
    with pytest.raises(RuntimeError, match="unsupported"):   # 61 x 3 16-bit samples: not whole 16-byte rows
        rs.Plan(64, 61, 3, 100, 100, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.bfloat16,
                flags=rs.RS_FORCE_STREAM)


def test_stream_unaligned_input_falls_back(rs):
    import torch

    H, W, C = 50, 64, 3
    img = synth.uniform(H, W, C, seed=21).astype(np.float32)
    want = oracle.resample(img.astype(np.float64), 70, 88, "lanczos", "mirror", param=3.0)
    p = rs.Plan(H, W, C, 70, 88, kernel="lanczos", boundary="mirror")
    assert p.path == "stream"
    flat = torch.zeros(H * W * C + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(img.reshape(-1)).cuda()
    out = torch.empty((70, 88, C), dtype=torch.float32, device="cuda")
    rs.rs_resample(p.handle, flat.data_ptr() + 4, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    p.check()
    assert np.abs(out.double().cpu().numpy() - want).max() <= TOL["f32"]
    p.close()


def test_stream_padded_pitches(rs):
    import torch

    H, W, C = 61, 50, 3
    img = synth.uniform(H, W, C, seed=5).astype(np.float32)
    want = oracle.resample(img.astype(np.float64), 83, 70, "cubic", "reflect101", param=-0.5)
    pitch_in, pitch_out = W * C + 10, 70 * C + 5           # 16-byte input pitch, odd output pitch
    src = torch.zeros((H, pitch_in), dtype=torch.float32, device="cuda")
    src[:, :W * C] = torch.from_numpy(img.reshape(H, W * C)).cuda()
    dst = torch.full((83, pitch_out), float("nan"), dtype=torch.float32, device="cuda")
    d = rs.make_desc(H, W, C, 83, 70, kernel="cubic", param=-0.5, boundary="reflect101", dtype=rs.RS_F32,
                     in_row_stride=pitch_in, out_row_stride=pitch_out, flags=rs.RS_FORCE_STREAM)
    h = rs.rs_plan_create(d, 0)
    assert rs.rs_plan_get_info(h).path == 3
    rs.rs_resample(h, src.data_ptr(), dst.data_ptr(), 0)
    torch.cuda.synchronize()
    rs.rs_plan_check(h)
    rs.rs_destroy(h)
    got = dst[:, :70 * C].double().cpu().numpy().reshape(83, 70, C)
    assert np.abs(got - want).max() <= TOL["f32"]
    assert torch.isnan(dst[:, 70 * C:]).all()


def test_stream_recompute_and_rerun(rs):
    import torch

    img = synth.sinusoids(300, 400, 3, seed=1)
    x = torch.from_numpy(img).cuda()
    p = rs.Plan(300, 400, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    assert p.path == "stream"
    a = p(x).clone()
    p.recompute()
    b = p(x).clone()
    torch.cuda.synchronize()
    p.check()
    p.close()
    assert torch.equal(a, b)
    want = oracle.resample(img.astype(np.float64), a.shape[0], a.shape[1], "lanczos", "mirror", param=3.0)
    assert np.abs(a.double().cpu().numpy() - want).max() <= TOL["f32"]


def test_stream_full_size_sampled_rows(rs):
    """4096x4096x3 x1.37 on the streaming kernel: sampled rows against the oracle."""
    t, exact = quantise(synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2), "f32")
    got, info = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, rs.RS_FORCE_STREAM, scale=1.37)
    assert info.path == 3 and (info.out_h, info.out_w) == (5612, 5612)
    g = np.random.default_rng(3)
    rows = sorted(set([0, 1, 2805, 2806, 5610, 5611]) | set(int(r) for r in g.integers(0, 5612, 10)))
    err = 0.0
    for r in rows:
        want = oracle.resample(exact, 5612, 5612, "lanczos", "mirror", param=3.0, rows=(r, r + 1))
        err = max(err, float(np.abs(got[r] - want[0]).max()))
    assert err <= TOL["f32"], err


def test_stream_full_size_x03_sampled_rows(rs):
    """4096x4096x3 x0.3 (antialiased, 20 taps) on the streaming kernel's wide strips."""
    t, exact = quantise(synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2), "f32")
    got, info = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, rs.RS_FORCE_STREAM, scale=0.3)
    assert info.path == 3 and (info.out_h, info.out_w) == (1229, 1229)
    g = np.random.default_rng(5)
    rows = sorted(set([0, 1, 614, 1227, 1228]) | set(int(r) for r in g.integers(0, 1229, 8)))
    err = 0.0
    for r in rows:
        want = oracle.resample(exact, 1229, 1229, "lanczos", "mirror", param=3.0, rows=(r, r + 1))
        err = max(err, float(np.abs(got[r] - want[0]).max()))
    assert err <= TOL["f32"], err


def test_autotune_chooses_between_stream_and_tiles(rs, tmp_path):
    import torch

    img = synth.sinusoids(700, 900, 3, seed=4)
    x = torch.from_numpy(img).cuda()
    cache = str(tmp_path / "tune.jsonl")
    p = rs.Plan(700, 900, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    out = torch.empty(p.out_shape, device="cuda")
    p.autotune(x, out, cache_path=cache)
    first = p.path
    assert first in ("stream", "fused", "two_pass")
    y = p(x)
    torch.cuda.synchronize()
    p.check()
    want = oracle.resample(img.astype(np.float64), p.info.out_h, p.info.out_w, "lanczos", "mirror", param=3.0)
    assert np.abs(y.double().cpu().numpy() - want).max() <= TOL["f32"]
    p.close()
    # a second plan takes the cached choice without timing
    q = rs.Plan(700, 900, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    q.autotune(x, out, cache_path=cache)
    assert q.path == first
    q.close()


# 16-bit rows must be whole 16-byte words (W * C a multiple of 8) for TMA
SHAPES16 = [((67, 96), (150, 203)),    # x2.2, ragged strips
            ((96, 136), (131, 181)),   # ~x1.37
            ((300, 400), (411, 548)),  # x1.37, several row ranges
            ((33, 40), (33, 40)),      # identity
            ((64, 104), (50, 77)),     # mild downscale
            ((40, 400), (90, 999)),    # wide, many strips
            ((200, 24), (401, 37)),    # tall, one strip
            ((300, 400), (90, 120)),   # x0.3: wide strips (two boxes per staged row)
            ((257, 616), (77, 183))]   # ~x0.3, ragged


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("shape", SHAPES16, ids=[f"{a[0]}x{a[1]}-{b[0]}x{b[1]}" for a, b in SHAPES16])
@pytest.mark.parametrize("kernel,param", [("linear", None), ("cubic", -0.5), ("lanczos", 3.0),
                                          ("bspline3", None)])
@pytest.mark.parametrize("boundary", ["clamp", "mirror", "reflect101", "truncate"])
@pytest.mark.parametrize("C", [1, 3])
def test_stream_parity_16bit(rs, dt, shape, kernel, param, boundary, C):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=(H * 37 + W * 11 + C) & 0xffff)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
    # forced streaming (a wide 16-bit downscale takes the tensor-core form, path
    # 5), and the SIMT streaming kernels alone (RS_FORCE_SIMT)
    for flags in (rs.RS_FORCE_STREAM, rs.RS_FORCE_STREAM | rs.RS_FORCE_SIMT):
        try:
            got, info = run_gpu(t, OH, OW, kernel, boundary, param, flags)
        except RuntimeError as e:
            assert "unsupported" in str(e) and OH < H, e
            continue
        assert info.path == 3 or (info.path == 5 and not flags & rs.RS_FORCE_SIMT and OH < H), info.path
        err = np.abs(got - want).max()
        assert err <= TOL[dt], (err, info.tile_w, flags)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_stream_16bit_matches_tile_kernel(rs, dt):
    """Both kernels filter in FP32 and round once: they agree to one rounding step."""
    img = synth.sinusoids(240, 320, 3, seed=9)
    t, exact = quantise(img, dt)
    a, ia = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, rs.RS_FORCE_STREAM, scale=1.37)
    b, ib = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, rs.RS_NO_STREAM | rs.RS_FORCE_SIMT, scale=1.37)
    assert (ia.path, ib.path) == (3, 0)
    ulp = 2.0 ** -8 if dt == "bf16" else 2.0 ** -11
    assert np.abs(a - b).max() <= ulp
    want = oracle.resample(exact, ia.out_h, ia.out_w, "lanczos", "mirror", param=3.0)
    assert np.abs(a - want).max() <= TOL[dt]


def test_stream_is_default_for_16bit_upscale(rs):
    import torch

    for dt in (torch.bfloat16, torch.float16):
        p = rs.Plan(4096, 4096, 3, scale=1.37, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt)
        assert p.path == "stream", (dt, p.path)
        p.close()
        # the wide antialiasing downscale takes the tensor-core streaming form,
        # forced streaming too; without the tensor cores the SIMT streaming kernel
        p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt)
        assert p.path == "tcstream", (dt, p.path)
        p.close()
        p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt,
                    flags=rs.RS_FORCE_STREAM)
        assert p.path == "tcstream", (dt, p.path)
        p.close()
        p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt,
                    flags=rs.RS_FORCE_STREAM | rs.RS_FORCE_SIMT)
        assert p.path == "stream", (dt, p.path)
        p.close()


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("scale,out,simt", [(1.37, 5612, 0), (0.3, 1229, 0), (0.3, 1229, 1)])
def test_stream_16bit_full_size_sampled_rows(rs, dt, scale, out, simt):
    """4096x4096x3 16-bit on the streaming kernels (x0.3: the tensor-core form,
    and the SIMT band kernel): sampled rows against the oracle."""
    t, exact = quantise(synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2), dt)
    flags = rs.RS_FORCE_STREAM | (rs.RS_FORCE_SIMT if simt else 0)
    got, info = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, flags, scale=scale)
    assert info.path == (5 if scale < 1 and not simt else 3) and (info.out_h, info.out_w) == (out, out)
    g = np.random.default_rng(7)
    rows = sorted(set([0, 1, out // 2, out - 2, out - 1]) | set(int(r) for r in g.integers(0, out, 8)))
    err = 0.0
    for r in rows:
        want = oracle.resample(exact, out, out, "lanczos", "mirror", param=3.0, rows=(r, r + 1))
        err = max(err, float(np.abs(got[r] - want[0]).max()))
    assert err <= TOL[dt], err


@pytest.mark.parametrize("env,want", [("NO_STREAM", "fused"), ("FORCE_SIMT, NO_STREAM", "fused"), ("", "stream"),
                                      ("BOGUS", "error")])
def test_plan_flags_environment(rs, env, want):
    """RS_PLAN_FLAGS adds kernel-choice flags to every plan of the process."""
    import os
    import subprocess
    import sys

    code = ("import paper_1110_5450_b300 as rs\n"
            "try:\n"
            "    p = rs.Plan(300, 400, 3, scale=1.37, kernel='lanczos', boundary='mirror')\n"
            "    print(p.path)\n"
            "except RuntimeError as e:\n"
            "    print('error' if 'RS_PLAN_FLAGS' in str(e) else str(e))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env_vars = dict(os.environ, RS_PLAN_FLAGS=env, PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env_vars, timeout=300)
    assert out.stdout.strip().splitlines()[-1] == want, out.stdout + out.stderr
