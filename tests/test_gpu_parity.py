"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (max-abs on [0, 1] data, the oracle fed the same quantised input):
FP32 2e-6, FP16 2e-3, BF16 1e-2; FP64 storage 1e-12.  Integer tap indices
are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import TOL, quantise, run_gpu

pytestmark = pytest.mark.gpu

KERNELS = [("linear", None), ("cubic", -0.5), ("lanczos", 3.0), ("bspline3", None)]
BOUNDARIES = ["clamp", "mirror", "reflect101", "truncate"]


@pytest.fixture(scope="module")
def rs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_5450_b300 as rs

    return rs


# ------------------------------------------------------------------ tables
GEOMS = [(256, 512), (4096, 5612), (4096, 1229), (4096, 512), (7, 3), (3, 7), (1, 5), (5, 1),
         (100, 37), (37, 100), (64, 32), (2, 2)]


@pytest.mark.parametrize("n_in,n_out", GEOMS)
@pytest.mark.parametrize("kernel,param", [("linear", None), ("cubic", -0.5), ("lanczos", 3.0),
                                          ("lanczos", 2.0)])
@pytest.mark.parametrize("aa", [True, False])
def test_tap_indices_bit_exact(rs, n_in, n_out, kernel, param, aa):
    import torch

    flags = 0 if aa else rs.RS_NO_ANTIALIAS
    p = rs.Plan(n_in, 4, 1, n_out, 4, kernel=kernel, param=param, boundary="clamp",
                dtype=torch.float32, flags=flags)
    jlo, cnt, start, w64, ww = p.tables(0)
    p.close()
    for i in range(n_out):
        jf, c = oracle.axis_taps(n_in, n_out, kernel, i, param=param, antialias=aa)
        assert (int(jlo[i]), int(cnt[i])) == (jf, c), (i, jlo[i], cnt[i], jf, c)


def _dense_oracle(n_in, n_out, kernel, boundary, param, aa=True):
    M = np.zeros((n_out, n_in))
    for i, (jf, idx, w) in enumerate(oracle.axis_weights(n_in, n_out, kernel, boundary, param, aa)):
        keep = idx >= 0
        np.add.at(M[i], idx[keep], w[keep])
    return M


def _dense_gpu(start, w, n_in):
    n_out, t = w.shape
    M = np.zeros((n_out, n_in))
    for i in range(n_out):
        M[i, start[i]:start[i] + t] = w[i]
    return M


@pytest.mark.parametrize("n_in,n_out", [(256, 512), (97, 41), (41, 97), (4096, 1229), (5, 2), (3, 9),
                                        (2, 50), (50, 2)])
@pytest.mark.parametrize("kernel,param", KERNELS)
@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_folded_weights_match_oracle(rs, n_in, n_out, kernel, param, boundary):
    import torch

    p = rs.Plan(n_in, 3, 1, n_out, 3, kernel=kernel, param=param, boundary=boundary,
                dtype=torch.float32)
    jlo, cnt, start, w64, ww = p.tables(0)
    p.close()
    assert np.all(start >= 0) and np.all(start + w64.shape[1] <= n_in)
    want = _dense_oracle(n_in, n_out, kernel, boundary, param)
    got = _dense_gpu(start, w64, n_in)
    assert np.abs(got - want).max() < 2e-15
    got32 = _dense_gpu(start, ww, n_in)
    assert np.abs(got32 - want).max() < 1.2e-7
    # the working-precision rows still sum to 1 after rounding (residual put back)
    assert np.abs(ww.sum(axis=1) - 1.0).max() < 2.5e-7


@pytest.mark.parametrize("n_in,n_out", [(4_000_000, 3_000_017), (4_000_000, 1_300_001), (1_234_567, 4_194_304)])
@pytest.mark.parametrize("kernel,param", [("lanczos", 3.0), ("lanczos", 16.0), ("cubic", -0.5)])
@pytest.mark.parametrize("boundary", ["mirror", "truncate"])
def test_long_axis_tables(rs, n_in, n_out, kernel, param, boundary):
    """Axes near the 2^22 side limit (tap numerators near 2^46, Lanczos
    argument numerators near 2^27): tap indices bit-exact and folded weights
    within the table tolerance on sampled outputs, both ends included."""
    import torch

    p = rs.Plan(n_in, 4, 1, n_out, 4, kernel=kernel, param=param, boundary=boundary, dtype=torch.float32)
    jlo, cnt, start, w64, ww = p.tables(0)
    p.close()
    g = np.random.default_rng(n_in + n_out)
    sample = sorted(set(range(40)) | set(range(n_out - 40, n_out)) | set(g.integers(0, n_out, 200).tolist()))
    te = w64.shape[1]
    for i in sample:
        jf, idx, w = oracle.axis_weights_at(n_in, n_out, kernel, boundary, i, param=param)
        assert (int(jlo[i]), int(cnt[i])) == (jf, len(idx)), i
        want = {}
        for m, v in zip(idx.tolist(), w.tolist()):
            if m >= 0:
                want[m] = want.get(m, 0.0) + v
        s0 = int(start[i])
        assert all(s0 <= m < s0 + te for m in want), i
        dense = np.zeros(te)
        for m, v in want.items():
            dense[m - s0] = v
        assert np.abs(w64[i] - dense).max() < 2e-15, i
        assert np.abs(ww[i].astype(np.float64) - dense).max() < 1.2e-7, i


def test_keys_x2_tables_exact(rs):
    """Keys a=-1/2 at x2: dyadic weights {-9, 111, 29, -3}/128 in FP64 and FP32."""
    import torch

    for dt in (torch.float64, torch.float32):
        p = rs.Plan(256, 256, 1, 512, 512, kernel="cubic", param=-0.5, boundary="clamp", dtype=dt)
        jlo, cnt, start, w64, ww = p.tables(0)
        p.close()
        for i in range(4, 508):
            want = np.array([-3, 29, 111, -9] if i % 2 == 0 else [-9, 111, 29, -3]) / 128.0
            assert np.array_equal(w64[i], want) and np.array_equal(ww[i], want), i


def test_recompute_reproduces_tables(rs):
    import torch

    p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", boundary="mirror", dtype=torch.float32)
    a = [p.tables(ax) for ax in (0, 1)]
    p.recompute()
    torch.cuda.synchronize()
    b = [p.tables(ax) for ax in (0, 1)]
    p.close()
    for ta, tb in zip(a, b):
        for x, y in zip(ta, tb):
            assert np.array_equal(x, y)


# ------------------------------------------------------------ small images
SHAPES = [((67, 91), (150, 203)),    # x2.2 up, several tiles + ragged tails
          ((96, 130), (131, 178)),   # ~x1.37
          ((200, 170), (61, 53)),    # ~x0.3, antialiased
          ((301, 257), (38, 33)),    # ~x0.125
          ((33, 33), (33, 33)),      # identity
          ((1, 1), (5, 3)),
          ((1, 40), (3, 9)),
          ((5, 4), (40, 2)),
          ((9, 300), (70, 30))]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a[0]}x{a[1]}-{b[0]}x{b[1]}" for a, b in SHAPES])
@pytest.mark.parametrize("kernel,param", KERNELS)
@pytest.mark.parametrize("boundary", BOUNDARIES)
@pytest.mark.parametrize("C", [1, 3])
def test_fp32_parity(rs, shape, kernel, param, boundary, C):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=hash((H, W, C)) & 0xffff)
    t, exact = quantise(img, "f32")
    want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
    for flags in (0, rs.RS_TWO_PASS):
        got, info = run_gpu(t, OH, OW, kernel, boundary, param, flags)
        err = np.abs(got - want).max()
        assert err <= TOL["f32"], (flags, info.path, err)


@pytest.mark.parametrize("dt", ["f64", "f16", "bf16"])
@pytest.mark.parametrize("shape", SHAPES[:4] + SHAPES[5:7], ids=lambda s: f"{s[0][0]}x{s[0][1]}-{s[1][0]}x{s[1][1]}")
@pytest.mark.parametrize("kernel,param", [("cubic", -0.5), ("lanczos", 3.0), ("linear", None)])
@pytest.mark.parametrize("C", [1, 3])
def test_other_dtypes_parity(rs, dt, shape, kernel, param, C):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=17)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, OH, OW, kernel, "mirror", param=param)
    for flags in (0, rs.RS_TWO_PASS):
        got, info = run_gpu(t, OH, OW, kernel, "mirror", param, flags)
        err = np.abs(got - want).max()
        assert err <= TOL[dt], (dt, flags, info.path, err)


@pytest.mark.parametrize("C", [2, 4, 5])
def test_other_channel_counts(rs, C):
    img = synth.uniform(40, 37, C, seed=5)
    t, exact = quantise(img, "f32")
    want = oracle.resample(exact, 29, 53, "lanczos", "reflect101", param=3.0)
    got, info = run_gpu(t, 29, 53, "lanczos", "reflect101", 3.0)
    assert np.abs(got - want).max() <= TOL["f32"]


def test_scale_derived_size(rs):
    img = synth.uniform(123, 77, 1, seed=9)
    t, exact = quantise(img, "f32")
    oh, ow = oracle.out_size(123, 0.61), oracle.out_size(77, 0.61)
    got, info = run_gpu(t, 0, 0, "cubic", "clamp", -0.5, scale=0.61)
    assert (info.out_h, info.out_w) == (oh, ow)
    want = oracle.resample(exact, oh, ow, "cubic", "clamp", param=-0.5)
    assert np.abs(got - want).max() <= TOL["f32"]


def test_no_antialias_flag(rs):
    img = synth.uniform(60, 60, 1, seed=3)
    t, exact = quantise(img, "f32")
    want = oracle.resample(exact, 19, 23, "cubic", "clamp", param=-0.75, antialias=False)
    got, _ = run_gpu(t, 19, 23, "cubic", "clamp", -0.75, rs.RS_NO_ANTIALIAS)
    assert np.abs(got - want).max() <= TOL["f32"]


def test_unaligned_input_pointer_and_strides(rs):
    """An input that is not 16-byte aligned (no TMA) and padded rows."""
    import torch

    H, W, C = 50, 61, 3
    img = synth.uniform(H, W, C, seed=21).astype(np.float32)
    want = oracle.resample(img.astype(np.float64), 70, 83, "lanczos", "mirror", param=3.0)
    flat = torch.zeros(H * W * C + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(img.reshape(-1)).cuda()
    p = rs.Plan(H, W, C, 70, 83, kernel="lanczos", boundary="mirror")
    out = torch.empty((70, 83, C), dtype=torch.float32, device="cuda")
    rs.rs_resample(p.handle, flat.data_ptr() + 4, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    p.check()
    assert np.abs(out.double().cpu().numpy() - want).max() <= TOL["f32"]
    p.close()
    # padded input and output rows
    pitch_in, pitch_out = W * C + 7, 83 * C + 5
    src = torch.zeros((H, pitch_in), dtype=torch.float32, device="cuda")
    src[:, :W * C] = torch.from_numpy(img.reshape(H, W * C)).cuda()
    dst = torch.full((70, pitch_out), float("nan"), dtype=torch.float32, device="cuda")
    d = rs.make_desc(H, W, C, 70, 83, kernel="lanczos", boundary="mirror", dtype=rs.RS_F32,
                     in_row_stride=pitch_in, out_row_stride=pitch_out)
    h = rs.rs_plan_create(d, 0)
    rs.rs_resample(h, src.data_ptr(), dst.data_ptr(), 0)
    torch.cuda.synchronize()
    rs.rs_plan_check(h)
    rs.rs_destroy(h)
    got = dst[:, :83 * C].double().cpu().numpy().reshape(70, 83, C)
    assert np.abs(got - want).max() <= TOL["f32"]
    assert torch.isnan(dst[:, 83 * C:]).all()


def test_deterministic_rerun(rs):
    import torch

    img = synth.sinusoids(300, 400, 3, seed=1)
    x = torch.from_numpy(img).cuda()
    p = rs.Plan(300, 400, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    a = p(x).clone()
    b = p(x).clone()
    torch.cuda.synchronize()
    p.close()
    assert torch.equal(a, b)


# ------------------------------------------------------- full-size configs
def test_c1_fp64_full(rs):
    """256x256 FP64 uniform, x2 with Keys a=-1/2, clamp, H then V (two-pass) and fused."""
    img = synth.uniform(256, 256, 1, seed=synth.SEED_C1)
    t, exact = quantise(img, "f64")
    want = oracle.resample(exact, 512, 512, "cubic", "clamp", param=-0.5)
    for flags in (rs.RS_TWO_PASS, 0):
        got, info = run_gpu(t, 512, 512, "cubic", "clamp", -0.5, flags)
        assert np.abs(got - want).max() <= TOL["f64"], flags
    t32, exact32 = quantise(img, "f32")
    want32 = oracle.resample(exact32, 512, 512, "cubic", "clamp", param=-0.5)
    got, _ = run_gpu(t32, 512, 512, "cubic", "clamp", -0.5)
    assert np.abs(got - want32).max() <= TOL["f32"]


def _sample_rows(n, k, seed):
    g = np.random.default_rng(seed)
    rows = set([0, 1, 2, n // 2, n - 2, n - 1]) | set(int(r) for r in g.integers(0, n, k))
    return sorted(r for r in rows if 0 <= r < n)


@pytest.fixture(scope="module")
def c2_image():
    return synth.sinusoids(4096, 4096, 3, seed=synth.SEED_C2)


@pytest.mark.parametrize("scale", [1.37, 0.3, 0.125])
@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_full_size_sampled_rows(rs, c2_image, scale, dt):
    """4096x4096x3 sinusoid+noise, Lanczos-3, mirror; the full output on the
    device, checked against the oracle on sampled rows (oracle row by row)."""
    t, exact = quantise(c2_image, dt)
    oh = ow = oracle.out_size(4096, scale)
    got, info = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, scale=scale)
    assert (info.out_h, info.out_w) == (oh, ow)
    rows = _sample_rows(oh, 10, 7)
    err = 0.0
    for r in rows:
        want = oracle.resample(exact, oh, ow, "lanczos", "mirror", param=3.0, rows=(r, r + 1))
        err = max(err, float(np.abs(got[r] - want[0]).max()))
    assert err <= TOL[dt], (scale, dt, err, info.path)
    assert np.isfinite(got).all()


def test_two_plans_sharing_a_kernel_variant(rs):
    """Plans of different shared-memory size on the same kernel variant,
    created one after the other and then used in either order."""
    import torch

    img = synth.sinusoids(512, 512, 3, seed=2)
    x = torch.from_numpy(img).cuda()
    a = rs.Plan(512, 512, 3, scale=1.37, kernel="lanczos", boundary="mirror")
    b = rs.Plan(512, 512, 3, scale=0.3, kernel="lanczos", boundary="mirror")
    ya, yb = a(x), b(x)
    torch.cuda.synchronize()
    for p, y in ((a, ya), (b, yb)):
        p.check()
        want = oracle.resample(img.astype(np.float64), p.info.out_h, p.info.out_w, "lanczos", "mirror",
                               param=3.0)
        assert np.abs(y.double().cpu().numpy() - want).max() <= TOL["f32"]
        p.close()


def test_fp64_autotune_times_the_two_pass_path(rs, tmp_path):
    """A small FP64 plan (256x256 -> 512x512, Keys): the autotuner also times
    the two-pass path; whichever wins keeps parity with the oracle, the
    recomputed tables give the same result, and a second plan takes the
    cached choice."""
    import torch

    img = synth.uniform(256, 256, 1, seed=synth.SEED_C1)
    x = torch.from_numpy(img).cuda()
    want = oracle.resample(img, 512, 512, "cubic", "clamp", param=-0.5)
    cache = str(tmp_path / "fp64.jsonl")
    paths = []
    for _ in range(2):
        p = rs.Plan(256, 256, 1, 512, 512, kernel="cubic", param=-0.5, boundary="clamp", dtype=torch.float64)
        out = torch.empty(p.out_shape, dtype=torch.float64, device="cuda")
        p.autotune(x, out, cache_path=cache)
        paths.append(p.path)
        y = p(x).clone()
        p.recompute()
        y2 = p(x)
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(y, y2)
        got = y.cpu().numpy()
        assert got.shape == want.shape
        assert np.abs(got - want).max() < 1e-13
        p.close()
    assert paths[0] == paths[1]
    assert '"two_pass":' in open(cache).read()


def test_autotune_keeps_parity_and_uses_cache(rs, tmp_path):
    import torch

    img = synth.sinusoids(700, 900, 3, seed=4)
    x = torch.from_numpy(img).cuda()
    cache = str(tmp_path / "tune.jsonl")
    p = rs.Plan(700, 900, 3, scale=0.61, kernel="lanczos", boundary="mirror")
    y = p.autotune(x, cache_path=cache)
    y = p(x, out=y)
    torch.cuda.synchronize()
    p.check()
    want = oracle.resample(img.astype(np.float64), p.info.out_h, p.info.out_w, "lanczos", "mirror", param=3.0)
    assert np.abs(y.double().cpu().numpy() - want).max() <= TOL["f32"]
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and '"G":' in lines[0]
    q = rs.Plan(700, 900, 3, scale=0.61, kernel="lanczos", boundary="mirror")
    q.autotune(x, cache_path=cache)
    assert (q.info.tile_h, q.info.tile_w, q.info.group_h, q.info.warps_pass1) == \
        (p.info.tile_h, p.info.tile_w, p.info.group_h, p.info.warps_pass1)
    assert len(open(cache).read().splitlines()) == 1  # a hit appends nothing
    z = q(x)
    torch.cuda.synchronize()
    assert torch.equal(y, z)
    p.close()
    q.close()
