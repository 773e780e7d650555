"""The tensor-core (tcgen05) vertical pass against the FP64 oracle.

The building block first: one-CTA tcgen05 GEMMs on host matrices against an
FP64 product of the same 16-bit values, for every operand major-ness.  Then
the fused kernel with its vertical pass on the tensor cores (plan path 2) on
BF16 / FP16 images, wide antialiased downscales (x0.3, x0.125) and, forced,
ordinary ones, element by element against the oracle fed the same quantised
input; tolerances FP16 2e-3, BF16 1e-2 (max-abs on [0, 1] data).
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


def _bits(x, bf16):
    """16-bit patterns of x (rounded to the type) and their exact float64 values."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16 if bf16 else torch.float16)
    return t.view(torch.int16).numpy().view(np.uint16), t.to(torch.float64).numpy()


@pytest.mark.parametrize("bf16", [1, 0])
@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("n,k", [(16, 16), (32, 80), (64, 256), (128, 96), (256, 64)])
def test_tc_selftest_gemm(rs, bf16, a_mn, b_mn, n, k):
    g = np.random.default_rng(n * 1000 + k)
    a16, a = _bits(g.uniform(-1, 1, (128, k)), bf16)
    b16, b = _bits(g.uniform(-1, 1, (n, k)), bf16)
    d = rs.rs_tc_selftest(a16, b16, a_mn=a_mn, b_mn=b_mn, variant=0, bf16=bf16)
    want = a @ b.T
    # FP32 accumulation of k exact products of 16-bit values
    assert np.abs(d - want).max() <= 1e-5 * k, (np.abs(d - want).max())


def test_tc_selftest_swapped_strides_differ(rs):
    """The check can tell the two stride encodings apart (K-major, k > 8)."""
    g = np.random.default_rng(3)
    a16, a = _bits(g.uniform(-1, 1, (128, 32)), 1)
    b16, b = _bits(g.uniform(-1, 1, (32, 32)), 1)
    d = rs.rs_tc_selftest(a16, b16, variant=1)
    assert np.abs(d - a @ b.T).max() > 1e-2


def test_tc_selftest_rejects_bad_shapes(rs):
    z = np.zeros((128, 24), np.uint16)
    with pytest.raises(RuntimeError):
        rs.rs_tc_selftest(z, np.zeros((16, 24), np.uint16))
    with pytest.raises(RuntimeError):
        rs.rs_tc_selftest(np.zeros((64, 16), np.uint16), np.zeros((16, 16), np.uint16))


# (H, W) with W * C a multiple of 8 for C in {1, 3}, outputs with ragged tiles
WIDE = [((200, 168), (60, 50)),     # ~x0.3
        ((304, 256), (38, 32)),     # x0.125
        ((211, 96), (23, 31)),      # ~x0.11 / x0.32, unequal axes
        ((64, 40), (19, 12))]       # ~x0.3, a single tile


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("shape", WIDE, ids=lambda s: f"{s[0][0]}x{s[0][1]}-{s[1][0]}x{s[1][1]}")
@pytest.mark.parametrize("kernel,param", [("lanczos", 3.0), ("cubic", -0.5), ("linear", None),
                                          ("bspline3", None)])
@pytest.mark.parametrize("boundary", ["mirror", "clamp", "reflect101", "truncate"])
@pytest.mark.parametrize("C", [1, 3])
def test_tc_parity_wide_downscale(rs, dt, shape, kernel, param, boundary, C):
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=H * 7 + W + C)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, OH, OW, kernel, boundary, param=param)
    got, info = run_gpu(t, OH, OW, kernel, boundary, param, rs.RS_FORCE_TC)
    assert info.path == 2
    err = np.abs(got - want).max()
    assert err <= TOL[dt], (err, info.tile_h, info.tile_w)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [((96, 128), (131, 176)), ((67, 88), (150, 200)), ((40, 48), (40, 48)),
                                   ((1, 8), (5, 3)), ((5, 16), (40, 2))],
                         ids=lambda s: f"{s[0][0]}x{s[0][1]}-{s[1][0]}x{s[1][1]}")
@pytest.mark.parametrize("C", [1, 3])
def test_tc_parity_forced_narrow(rs, dt, shape, C):
    """Upscales, identity and degenerate sizes forced onto the tensor cores."""
    (H, W), (OH, OW) = shape
    img = synth.uniform(H, W, C, seed=11)
    t, exact = quantise(img, dt)
    want = oracle.resample(exact, OH, OW, "lanczos", "mirror", param=3.0)
    got, info = run_gpu(t, OH, OW, "lanczos", "mirror", 3.0, rs.RS_FORCE_TC)
    assert info.path == 2
    assert np.abs(got - want).max() <= TOL[dt]


def test_tc_chosen_automatically_for_wide_16bit(rs):
    import torch

    for dt in (torch.bfloat16, torch.float16):
        for s in (0.3, 0.125):
            # the tensor-core streaming downscale; its fused tiles when forced
            p = rs.Plan(4096, 4096, 3, scale=s, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt)
            assert p.path == "tcstream", (dt, s, p.path)
            p.close()
            p = rs.Plan(4096, 4096, 3, scale=s, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt,
                        flags=rs.RS_FORCE_TC)
            assert p.path == "tcgen05", (dt, s, p.path)
            p.close()
        # narrow: the SIMT streaming kernel
        p = rs.Plan(4096, 4096, 3, scale=1.37, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt)
        assert p.path == "stream"
        p.close()
        p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt,
                    flags=rs.RS_FORCE_SIMT)
        assert p.path == "stream"
        p.close()
        p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=dt,
                    flags=rs.RS_FORCE_SIMT | rs.RS_NO_STREAM)
        assert p.path == "fused"
        p.close()
    p = rs.Plan(4096, 4096, 3, scale=0.3, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float32)
    assert p.path in ("fused", "stream")   # FP32 never takes the 16-bit tensor-core path
    p.close()


def test_force_tc_rejected_where_unsupported(rs):
    import torch

    with pytest.raises(RuntimeError, match="unsupported"):
        rs.Plan(64, 64, 1, 20, 20, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float32,
                flags=rs.RS_FORCE_TC)
    with pytest.raises(RuntimeError, match="unsupported"):   # 61 * 3 samples per row: not whole chunks
        rs.Plan(64, 61, 3, 20, 20, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.bfloat16,
                flags=rs.RS_FORCE_TC)


def test_tc_rejects_misaligned_input(rs):
    import torch

    p = rs.Plan(64, 64, 1, 20, 20, kernel="lanczos", param=3.0, boundary="mirror", dtype=torch.float16,
                flags=rs.RS_FORCE_TC)
    buf = torch.zeros(64 * 64 + 8, dtype=torch.float16, device="cuda")
    out = torch.empty((20, 20, 1), dtype=torch.float16, device="cuda")
    with pytest.raises(RuntimeError, match="invalid argument"):
        rs.rs_resample(p.handle, buf.data_ptr() + 2, out.data_ptr(), 0)
    p.close()


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_tc_matches_simt_path(rs, dt):
    """Both paths of one wide downscale stay within the tolerance of each other."""
    img = synth.sinusoids(480, 640, 3, seed=8)
    t, exact = quantise(img, dt)
    a, ia = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, 0, scale=0.3)
    b, ib = run_gpu(t, 0, 0, "lanczos", "mirror", 3.0, rs.RS_FORCE_SIMT | rs.RS_NO_STREAM, scale=0.3)
    assert (ia.path, ib.path) == (5, 0)
    assert np.abs(a - b).max() <= TOL[dt]
    want = oracle.resample(exact, ia.out_h, ia.out_w, "lanczos", "mirror", param=3.0)
    assert np.abs(a - want).max() <= TOL[dt]


@pytest.mark.parametrize("forced", [0, 1])
def test_tc_autotune_keeps_parity(rs, tmp_path, forced):
    """Autotuning a tensor-core plan times it against the SIMT kernels (unless
    the tensor cores are forced) and keeps parity whichever wins; a second plan
    takes the cached choice."""
    import torch

    img = synth.sinusoids(600, 800, 3, seed=6)
    t, exact = quantise(img, "bf16")
    x = t.cuda()
    flags = rs.RS_FORCE_TC if forced else 0
    cache = str(tmp_path / "tc.jsonl")
    want = None
    paths = []
    for _ in range(2):
        p = rs.Plan(600, 800, 3, scale=0.125, kernel="lanczos", param=3.0, boundary="mirror",
                    dtype=torch.bfloat16, flags=flags)
        assert p.path == ("tcgen05" if forced else "tcstream")
        out = torch.empty((p.info.out_h, p.info.out_w, 3), dtype=torch.bfloat16, device="cuda")
        p.autotune(x, out, cache_path=cache)
        paths.append(p.path)
        if forced:
            assert p.path == "tcgen05"
        y = p(x)
        torch.cuda.synchronize()
        p.check()
        if want is None:
            want = oracle.resample(exact, p.info.out_h, p.info.out_w, "lanczos", "mirror", param=3.0)
        assert np.abs(y.double().cpu().numpy() - want).max() <= TOL["bf16"]
        p.close()
    assert paths[0] == paths[1]
