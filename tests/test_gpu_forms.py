"""Every form of the row-streaming kernel, forced through the C ABI
(rs_plan_set_stream_form), against the FP64 oracle; and the very plans the
benchmark times (4096x4096x3, Lanczos-3, mirror, autotuned exactly as
bench.py tunes them) on sampled rows.

Forms: the band kernel with alternating phases (2 or 3 staged blocks), the
band kernel with warps specialised on the passes (3, 4 or 5 horizontal warps x
2 or 3 staged blocks), and the pipelined kernel (1 to 4 horizontal warps, 2
or 3 staged blocks, 3 to 8 vertical warps -- CTAs of more than 12 warps take
a whole SM --, with and without the L2 prefetch), each at the cost
model's strip width and at explicit narrow and wide widths.  Tolerances FP32
2e-6, FP16 2e-3, BF16 1e-2 (max-abs on [0, 1] data, the oracle fed the same
quantised input).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TOL, quantise, torch_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_5450_b300 as rs

    return rs


# (kind, horizontal warps, staged blocks, prefetch, vertical warps of kind 2)
FORMS = [(0, 0, 2, 0, 0), (0, 0, 3, 0, 0),
         (1, 3, 2, 0, 0), (1, 3, 3, 0, 0), (1, 4, 2, 0, 0), (1, 4, 3, 0, 0), (1, 5, 2, 0, 0), (1, 5, 3, 0, 0),
         (2, 1, 2, 0, 0), (2, 2, 2, 0, 0), (2, 3, 2, 0, 0), (2, 3, 3, 0, 0), (2, 4, 2, 0, 4), (2, 3, 2, 1, 0),
         (2, 4, 2, 0, 3), (2, 7, 2, 0, 8), (2, 5, 3, 1, 6)]
FORM_IDS = ["k%d-h%d-s%d%s%s" % (k, h, s, "-pf" if pf else "", "-v%d" % vw if vw else "")
            for k, h, s, pf, vw in FORMS]

# (every input row a whole number of 16-byte words: the streaming kernels stage rows by TMA)
SHAPES = [((96, 132), (131, 181)),    # ~x1.37
          ((300, 400), (411, 548)),   # x1.37, several row ranges
          ((67, 92), (150, 203)),     # x2.2, ragged strips
          ((33, 36), (33, 36)),       # identity
          ((257, 612), (77, 183))]    # ~x0.3: band kernels only
SHAPE_IDS = ["%dx%d-%dx%d" % (a[0], a[1], b[0], b[1]) for a, b in SHAPES]


def _resample_with_form(rs, t, OH, OW, kernel, boundary, param, form, width):
    """(result as float64 numpy, the form read back), or None when the plan
    cannot take the form at this strip width."""
    import torch

    kind, hw, ns, pf, vw = form
    H, W, C = t.shape
    x = t.to("cuda").contiguous()
    p = rs.Plan(H, W, C, OH, OW, kernel=kernel, param=param, boundary=boundary, dtype=x.dtype)
    try:
        try:
            rs.rs_plan_set_stream_form(p.handle, kind, hw, ns, width, pf,
                                       torch.cuda.current_stream().cuda_stream, vw)
        except rs.RSError as e:
            assert e.status == rs.RS_ERR_UNSUPPORTED, e
            return None
        p.info = rs.rs_plan_get_info(p.handle)
        assert p.info.path == 3
        got_form = rs.rs_plan_get_stream_form(p.handle)
        assert (got_form.kind, got_form.prefetch) == (kind, pf)
        if kind == 2 and vw:
            assert got_form.v_warps == vw
        if width:
            assert got_form.strip_width == width
        y = p(x)
        torch.cuda.synchronize()
        p.check()
        return y.to(torch.float64).cpu().numpy(), got_form
    finally:
        p.close()


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("kernel,param", [("cubic", -0.5), ("lanczos", 3.0)])
@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("width", [0, 16, 40])
def test_every_form_fp32(rs, form, shape, kernel, param, C, width):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=(H * 13 + W * 5 + C) & 0xffff)
    t, exact = quantise(img, "f32")
    want = oracle.resample(exact, OH, OW, kernel, "mirror", param=param)
    r = _resample_with_form(rs, t, OH, OW, kernel, "mirror", param, form, width)
    if r is None:
        # the pipelined kernel takes upscales (and identity) only; the band
        # kernels refuse only widths whose staged rows do not fit
        assert form[0] != 2 or OH < H or width, (form, shape, width)
        return
    got, _ = r
    err = np.abs(got - want).max()
    assert err <= TOL["f32"], (form, width, err)


@pytest.mark.parametrize("form", [f for f in FORMS if f[0] == 2], ids=[i for f, i in zip(FORMS, FORM_IDS) if f[0] == 2])
@pytest.mark.parametrize("boundary", ["clamp", "reflect101", "truncate"])
@pytest.mark.parametrize("kernel,param", [("bspline3", None), ("mitchell", 1.0 / 3.0), ("lanczos", 2.0)])
def test_exact_form_kernels_and_boundaries(rs, form, boundary, kernel, param):
    """The pipelined kernel with the other 4-tap kernels and boundaries."""
    img = synth.uniform(70, 92, 3, seed=77)     # rows of 1104 bytes: a 16-byte pitch
    t, exact = quantise(img, "f32")
    want = oracle.resample(exact, 113, 151, kernel, boundary, param=param)
    r = _resample_with_form(rs, t, 113, 151, kernel, boundary, param, form, 0)
    if r is None:
        # truncate keeps partial windows at the edges: those plans may not be eligible
        assert boundary == "truncate", (form, boundary, kernel)
        return
    got, _ = r
    assert np.abs(got - want).max() <= TOL["f32"]


@pytest.mark.parametrize("dt", ["f16", "bf16"])
@pytest.mark.parametrize("form", [(0, 0, 2, 0, 0), (1, 4, 3, 0, 0), (2, 3, 2, 0, 0), (2, 2, 3, 1, 5),
                                  (2, 7, 2, 0, 8)],
                         ids=["k0", "k1", "k2", "k2-pf", "k2-big"])
@pytest.mark.parametrize("C", [1, 3])
def test_forms_16bit(rs, dt, form, C):
    img = synth.uniform(96, 136, C, seed=9 + C)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, 131, 186, "lanczos", "mirror", param=3.0)
    r = _resample_with_form(rs, t, 131, 186, "lanczos", "mirror", 3.0, form, 0)
    assert r is not None, form
    got, _ = r
    assert np.abs(got - want).max() <= TOL[dt]


def test_form_is_reported_and_refused_cleanly(rs):
    import torch

    p = rs.Plan(256, 256, 3, scale=0.3, kernel="lanczos", boundary="mirror")
    s = torch.cuda.current_stream().cuda_stream
    before = rs.rs_plan_get_info(p.handle).path
    with pytest.raises(rs.RSError) as e:      # x0.3 is no upscale
        rs.rs_plan_set_stream_form(p.handle, 2, 0, 0, 0, 0, s)
    assert e.value.status == rs.RS_ERR_UNSUPPORTED
    assert rs.rs_plan_get_info(p.handle).path == before
    with pytest.raises(rs.RSError) as e:      # malformed
        rs.rs_plan_set_stream_form(p.handle, 4, 0, 0, 0, 0, s)
    assert e.value.status == rs.RS_ERR_INVALID_ARG
    with pytest.raises(rs.RSError) as e:
        rs.rs_plan_set_stream_form(p.handle, 1, 0, 0, 18, 0, s)  # width not a multiple of 4
    assert e.value.status == rs.RS_ERR_INVALID_ARG
    p.close()
    q = rs.Plan(256, 256, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    f = rs.rs_plan_get_stream_form(q.handle)
    assert f.kind == 2 and q.path == "stream"   # the untuned default for an FP32 Lanczos-3 upscale
    q.close()


def _sample_rows(n, k, seed):
    g = np.random.default_rng(seed)
    rows = set([0, 1, 2, n // 2, n - 2, n - 1]) | set(int(r) for r in g.integers(0, n, k))
    return sorted(r for r in rows if 0 <= r < n)


@pytest.fixture(scope="module")
def c2_image():
    return synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2)


@pytest.mark.parametrize("dt,scale", [("f32", 1.37), ("f32", 0.3), ("f16", 0.3), ("bf16", 0.3),
                                      ("f16", 0.125), ("bf16", 0.125), ("bf16", 1.37)])
def test_benchmarked_plans_autotuned(rs, c2_image, dt, scale):
    """The benchmark's plans: 4096x4096x3 Lanczos-3 mirror, autotuned on their
    own buffers as bench.py does, then the timed call (tables recomputed,
    resample) checked on sampled rows against the oracle."""
    import torch

    t, exact = quantise(c2_image, dt)
    x = t.to("cuda").contiguous()
    p = rs.Plan(4096, 4096, 3, scale=scale, kernel="lanczos", param=3.0, boundary="mirror",
                dtype=torch_dtype(dt))
    y = torch.empty(p.out_shape, dtype=x.dtype, device="cuda")
    p.autotune(x, out=y)
    y.fill_(float("nan"))
    p.recompute()
    p(x, out=y)
    torch.cuda.synchronize()
    p.check()
    oh, ow = p.info.out_h, p.info.out_w
    err = 0.0
    for r in _sample_rows(oh, 10, 17):
        want = oracle.resample(exact, oh, ow, "lanczos", "mirror", param=3.0, rows=(r, r + 1))
        err = max(err, float(np.abs(y[r].double().cpu().numpy() - want[0]).max()))
    assert err <= TOL[dt], (dt, scale, err, p.path)
    assert torch.isfinite(y).all()
    p.close()
