"""The FP32 streaming downscale (stream form 4, plan path 6): horizontal
bands of 4 outputs summed on SIMT warps from TMA-staged rows into a ring of
filtered rows, the vertical pass over groups of 4 output rows.  Checked
against the FP64 oracle at the FP32 tolerance: ragged strips and row runs, 1
and 3 channels, several warp and staged-block counts, the boundary rules,
recomputed tables, and the refusals."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_5450_b300 as rs

    return rs


def _run(rs, img, OH, OW, kernel, param, boundary, form=(0, 0, 0)):
    """(result float64, oracle, plan info) with stream form 4 forced
    (horizontal warps, staged blocks, vertical warps; 0 = default)."""
    import torch

    H, W, C = img.shape
    x = torch.from_numpy(np.ascontiguousarray(img)).to(torch.float32)
    exact = x.double().numpy()
    x = x.to("cuda").contiguous()
    p = rs.Plan(H, W, C, OH, OW, kernel=kernel, param=param, boundary=boundary, dtype=torch.float32)
    try:
        rs.rs_plan_set_stream_form(p.handle, 4, form[0], form[1], 0, 0, torch.cuda.current_stream().cuda_stream,
                                   form[2])
        p.info = rs.rs_plan_get_info(p.handle)
        assert p.path == "fstream"
        f = rs.rs_plan_get_stream_form(p.handle)
        assert f.kind == 4 and f.strip_width == 48 // C
        for got, asked in zip((f.h_warps, f.staged_blocks, f.v_warps), form):
            if asked:
                assert got == asked
        y = p(x)
        torch.cuda.synchronize()
        p.check()
        want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
        return y.double().cpu().numpy(), want, p.info
    finally:
        p.close()


SHAPES = [((600, 640), (180, 192)),     # x0.3
          ((520, 512), (65, 154)),      # x0.125 down, x0.3 across
          ((333, 408), (200, 245)),     # x0.6, ragged last strip
          ((1000, 96), (299, 29)),      # tall: several blocks per run, one strip
          ((129, 2044), (40, 600))]     # one block of rows, many strips
SHAPE_IDS = ["%dx%d-%dx%d" % (a[0], a[1], b[0], b[1]) for a, b in SHAPES]


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("kernel,param", [("lanczos", 3.0), ("cubic", -0.5)])
def test_fstream_matches_oracle(rs, shape, C, kernel, param):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=(H * 5 + W + C) & 0xffff)
    got, want, _ = _run(rs, img, OH, OW, kernel, param, "mirror")
    err = np.abs(got - want).max()
    assert err <= TOL["f32"], (shape, C, kernel, err)


@pytest.mark.parametrize("form", [(6, 2, 6), (6, 3, 6), (6, 4, 6), (6, 5, 4), (1, 4, 6), (4, 4, 4), (8, 4, 10),
                                  (6, 4, 1), (2, 2, 8), (10, 3, 8), (12, 3, 6), (8, 2, 10)],
                         ids=lambda f: "hw%d-na%d-vw%d" % f)
def test_fstream_forms(rs, form):
    """Every warp split, including those whose horizontal warps step
    ceil(HW / 4) = NA staged blocks per task, across the strip changes of
    the CTAs' runs."""
    img = synth.uniform(700, 768, 3, seed=23)
    got, want, _ = _run(rs, img, 210, 230, "lanczos", 3.0, "mirror", form=form)
    assert np.abs(got - want).max() <= TOL["f32"], form


@pytest.mark.parametrize("boundary", ["clamp", "reflect101", "truncate"])
def test_fstream_boundaries(rs, boundary):
    img = synth.uniform(400, 512, 3, seed=35)
    got, want, _ = _run(rs, img, 120, 150, "lanczos", 3.0, boundary)
    assert np.abs(got - want).max() <= TOL["f32"], boundary


def test_fstream_recompute(rs):
    """The kernel reads the plan's weight tables directly: recomputed tables
    give the same result."""
    import torch

    img = synth.sinusoids(512, 768, 3, seed=7)
    x = torch.from_numpy(img).to(torch.float32)
    exact = x.double().numpy()
    x = x.to("cuda").contiguous()
    p = rs.Plan(512, 768, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float32)
    rs.rs_plan_set_stream_form(p.handle, 4, 0, 0, 0, 0, torch.cuda.current_stream().cuda_stream, 0)
    y0 = p(x)
    p.recompute()
    y1 = p(x)
    torch.cuda.synchronize()
    p.check()
    assert torch.equal(y0, y1)
    want = oracle.resample(exact, p.out_shape[0], p.out_shape[1], "lanczos", "mirror", param=3.0)
    assert np.abs(y1.double().cpu().numpy() - want).max() <= TOL["f32"]
    p.close()


def test_fstream_refusals(rs):
    import torch

    s = torch.cuda.current_stream().cuda_stream
    cases = [dict(in_h=256, in_w=256, channels=3, scale=0.3, dtype=torch.bfloat16),  # 16-bit
             dict(in_h=256, in_w=256, channels=3, scale=1.5, dtype=torch.float32),   # an upscale
             dict(in_h=256, in_w=256, channels=3, scale=0.1, dtype=torch.float32),   # 60 taps across
             dict(in_h=256, in_w=256, channels=4, scale=0.3, dtype=torch.float32)]   # 4 channels
    for c in cases:
        p = rs.Plan(c["in_h"], c["in_w"], c["channels"], scale=c["scale"], kernel="lanczos", param=3.0,
                    boundary="mirror", dtype=c["dtype"])
        before = p.path
        with pytest.raises(rs.RSError) as e:
            rs.rs_plan_set_stream_form(p.handle, 4, 0, 0, 0, 0, s)
        assert e.value.status == rs.RS_ERR_UNSUPPORTED, c
        assert rs.PATHS[rs.rs_plan_get_info(p.handle).path] == before
        p.close()
    p = rs.Plan(256, 256, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float32)
    for bad in [dict(h_warps=13), dict(staged_blocks=1), dict(staged_blocks=7), dict(v_warps=11),
                dict(strip_width=16), dict(prefetch=1)]:
        args = dict(h_warps=0, staged_blocks=0, strip_width=0, prefetch=0, v_warps=0)
        args.update(bad)
        with pytest.raises(rs.RSError) as e:
            rs.rs_plan_set_stream_form(p.handle, 4, args["h_warps"], args["staged_blocks"], args["strip_width"],
                                       args["prefetch"], s, args["v_warps"])
        assert e.value.status == rs.RS_ERR_INVALID_ARG, bad
    # 12 horizontal warps step 3 staged blocks per task: more than 2 stages hold
    with pytest.raises(rs.RSError) as e:
        rs.rs_plan_set_stream_form(p.handle, 4, 12, 2, 0, 0, s, 6)
    assert e.value.status == rs.RS_ERR_UNSUPPORTED
    p.close()


@pytest.mark.parametrize("vw", [6, 10])
def test_fstream_runs_of_several_blocks(rs, vw):
    """Runs of a few blocks where some vertical warps have no output rows:
    every block must still be released in order."""
    img = synth.uniform(2048, 1024, 3, seed=46)
    got, want, _ = _run(rs, img, 256, 300, "lanczos", 3.0, "mirror", form=(0, 0, vw))
    assert np.abs(got - want).max() <= TOL["f32"]


def test_fstream_full_size_x03_against_band_kernel(rs):
    """4096x4096x3 x0.3, Lanczos-3 (20 taps): the default plan (this form) on
    sampled rows against the oracle, and bit for bit against the warp-specialised
    band kernel (the same taps in the same order: horizontal bands of 4 outputs
    from 4-pixel aligned bases, vertical bands of 4 rows from the first row's
    window start, zero weights adding exact zeros)."""
    import torch

    img = synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2)
    x32 = torch.from_numpy(img).to(torch.float32)
    exact = x32.double().numpy()
    x = x32.to("cuda").contiguous()
    s = torch.cuda.current_stream().cuda_stream
    p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float32)
    try:
        assert p.path == "fstream", p.path
        y = p(x).clone()
        rs.rs_plan_set_stream_form(p.handle, 1, 5, 2, 16, 0, s)
        p.info = rs.rs_plan_get_info(p.handle)
        assert p.path == "stream"
        yb = p(x)
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(y, yb)
    finally:
        p.close()
    got = y.double().cpu().numpy()
    g = np.random.default_rng(9)
    rows = sorted(set([0, 1, 614, 1227, 1228]) | set(int(r) for r in g.integers(0, 1229, 6)))
    err = 0.0
    for r in rows:
        want = oracle.resample(exact, 1229, 1229, "lanczos", "mirror", param=3.0, rows=(r, r + 1))
        err = max(err, float(np.abs(got[r] - want[0]).max()))
    assert err <= TOL["f32"], err
