"""The tensor-core streaming downscale (stream form 3, plan path 5): the
horizontal pass as a tcgen05 GEMM against each strip's weight matrix, the
vertical pass in FP32 on the rows read back from tensor memory.  Checked
against the FP64 oracle (fed the same quantised input) at the 16-bit
tolerances: ragged strips and row runs, 1 and 3 channels, every staged-chunk
count and several vertical-warp counts, the boundary rules, recomputed
tables, and the refusals."""
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


def _run(rs, img, dt, OH, OW, kernel, param, boundary, form=(0, 0), flags=0):
    """(result float64, plan info, form) with stream form 3 forced (staged chunks, vertical warps)."""
    import torch

    H, W, C = img.shape
    t, exact = quantise(img, dt)
    x = t.to("cuda").contiguous()
    p = rs.Plan(H, W, C, OH, OW, kernel=kernel, param=param, boundary=boundary, dtype=torch_dtype(dt), flags=flags)
    try:
        rs.rs_plan_set_stream_form(p.handle, 3, 0, form[0], 0, 0, torch.cuda.current_stream().cuda_stream,
                                   form[1])
        p.info = rs.rs_plan_get_info(p.handle)
        assert p.path == "tcstream"
        f = rs.rs_plan_get_stream_form(p.handle)
        assert f.kind == 3 and f.strip_width == 48 // C
        if form[0]:
            assert f.staged_blocks == form[0]
        if form[1]:
            assert f.v_warps == form[1]
        y = p(x)
        torch.cuda.synchronize()
        p.check()
        want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
        return y.double().cpu().numpy(), want, p.info
    finally:
        p.close()


SHAPES = [((600, 640), (180, 192)),     # x0.3
          ((520, 1024), (65, 128)),     # x0.125 across and down
          ((333, 408), (200, 245)),     # x0.6, ragged last strip
          ((1000, 96), (299, 29)),      # tall: several blocks per run, one strip
          ((129, 2048), (40, 600))]     # one block of rows, many strips
SHAPE_IDS = ["%dx%d-%dx%d" % (a[0], a[1], b[0], b[1]) for a, b in SHAPES]


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("kernel,param", [("lanczos", 3.0), ("cubic", -0.5)])
def test_tcstream_matches_oracle(rs, shape, C, dt, kernel, param):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=(H * 7 + W + C) & 0xffff)
    got, want, _ = _run(rs, img, dt, OH, OW, kernel, param, "mirror")
    err = np.abs(got - want).max()
    assert err <= TOL[dt], (shape, C, dt, kernel, err)


@pytest.mark.parametrize("form", [(2, 4), (3, 4), (4, 4), (5, 4), (6, 4), (4, 1), (4, 2), (4, 6), (4, 8), (4, 10)],
                         ids=lambda f: "na%d-vw%d" % f)
def test_tcstream_forms(rs, form):
    img = synth.uniform(700, 768, 3, seed=21)
    got, want, info = _run(rs, img, "bf16", 210, 230, "lanczos", 3.0, "mirror", form=form)
    assert np.abs(got - want).max() <= TOL["bf16"], form


@pytest.mark.parametrize("boundary", ["clamp", "reflect101", "truncate"])
def test_tcstream_boundaries(rs, boundary):
    img = synth.uniform(400, 512, 3, seed=33)
    got, want, _ = _run(rs, img, "f16", 120, 150, "lanczos", 3.0, boundary)
    assert np.abs(got - want).max() <= TOL["f16"], boundary


def test_tcstream_recompute_and_default(rs):
    """Recomputed tables rebuild the strips' weight matrices (same result), and
    an untuned 16-bit downscale plan runs this form."""
    import torch

    img = synth.sinusoids(512, 768, 3, seed=5)
    t, exact = quantise(img, "bf16")
    x = t.to("cuda").contiguous()
    p = rs.Plan(512, 768, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.bfloat16)
    assert p.path == "tcstream", p.path
    y0 = p(x)
    p.recompute()
    y1 = p(x)
    torch.cuda.synchronize()
    p.check()
    assert torch.equal(y0, y1)
    want = oracle.resample(exact, p.out_shape[0], p.out_shape[1], "lanczos", "mirror", param=3.0)
    assert np.abs(y1.double().cpu().numpy() - want).max() <= TOL["bf16"]
    p.close()


def test_tcstream_refusals(rs):
    import torch

    s = torch.cuda.current_stream().cuda_stream
    cases = [dict(in_h=256, in_w=256, channels=3, scale=0.3, dtype=torch.float32),   # FP32
             dict(in_h=256, in_w=256, channels=3, scale=1.5, dtype=torch.bfloat16),  # an upscale
             dict(in_h=256, in_w=250, channels=3, scale=0.3, dtype=torch.bfloat16)]  # in_w * C not a multiple of 8
    for c in cases:
        p = rs.Plan(c["in_h"], c["in_w"], c["channels"], scale=c["scale"], kernel="lanczos", param=3.0,
                    boundary="mirror", dtype=c["dtype"])
        before = p.path
        with pytest.raises(rs.RSError) as e:
            rs.rs_plan_set_stream_form(p.handle, 3, 0, 0, 0, 0, s)
        assert e.value.status == rs.RS_ERR_UNSUPPORTED, c
        assert rs.PATHS[rs.rs_plan_get_info(p.handle).path] == before
        p.close()
    p = rs.Plan(256, 256, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.bfloat16)
    for bad in [dict(h_warps=1), dict(staged_blocks=1), dict(staged_blocks=7), dict(v_warps=11), dict(strip_width=16)]:
        args = dict(h_warps=0, staged_blocks=0, strip_width=0, prefetch=0, v_warps=0)
        args.update(bad)
        with pytest.raises(rs.RSError) as e:
            rs.rs_plan_set_stream_form(p.handle, 3, args["h_warps"], args["staged_blocks"], args["strip_width"],
                                       args["prefetch"], s, args["v_warps"])
        assert e.value.status == rs.RS_ERR_INVALID_ARG, bad
    p.close()


@pytest.mark.parametrize("vw", [8, 10])
def test_tcstream_runs_of_several_blocks(rs, vw):
    """Runs of a few blocks where some vertical warps have no output rows
    (x0.125: 28 output rows per CTA over 3 blocks of input rows, 7 groups of
    4 rows for up to 10 warps): every block must still be released in order."""
    img = synth.uniform(2048, 2048, 3, seed=44)
    got, want, _ = _run(rs, img, "bf16", 256, 256, "lanczos", 3.0, "mirror", form=(0, vw))
    assert np.abs(got - want).max() <= TOL["bf16"]
