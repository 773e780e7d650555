"""Batched path: uneven images in one persistent launch (CUDA graph),
checked image by image against the FP64 oracle and against the
single-image path (bit-identical: the zero-padded weight bands add exact
zeros in the same order whatever the tile configuration)."""
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


def _specs(n, seed, side=(17, 300)):
    g = np.random.default_rng(seed)
    kernels = [("linear", None), ("cubic", -0.5), ("lanczos", 3.0)]
    out = []
    for i in range(n):
        k, p = kernels[i % 3]
        out.append(dict(in_h=int(g.integers(*side)), in_w=int(g.integers(*side)),
                        scale=float(np.exp(g.uniform(np.log(0.25), np.log(4.0)))), kernel=k, param=p,
                        boundary=["mirror", "clamp", "reflect101", "truncate"][i % 4]))
    return out


def _run_batch(rs, specs, C, dt, aligned):
    import torch

    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dt]
    elem = 4 if dt == "f32" else 2
    vec = 16 // elem
    ins, exact, pitches, outs = [], [], [], []
    for i, sp in enumerate(specs):
        img = synth.sinusoids(sp["in_h"], sp["in_w"], C, seed=1000 + i)
        t = torch.from_numpy(img).to(tdt)
        exact.append(t.double().numpy())
        row = sp["in_w"] * C
        pitch = ((row + vec - 1) // vec) * vec if aligned else row
        buf = torch.zeros((sp["in_h"], pitch), dtype=tdt, device="cuda")
        buf[:, :row] = t.reshape(sp["in_h"], row).cuda()
        ins.append(buf)
        pitches.append(pitch)
    b = rs.Batch(specs, channels=C, dtype=tdt, in_pitches=pitches)
    for i, sp in enumerate(specs):
        oh, ow = oracle.out_size(sp["in_h"], sp["scale"]), oracle.out_size(sp["in_w"], sp["scale"])
        outs.append(torch.full((oh, ow, C), float("nan"), dtype=tdt, device="cuda"))
    return b, ins, outs, exact, pitches


@pytest.mark.parametrize("dt,C,aligned", [("f32", 1, False), ("f16", 1, True), ("bf16", 3, True),
                                          ("f32", 3, True), ("f16", 1, False)])
def test_batch_matches_oracle_and_single_path(rs, dt, C, aligned):
    import torch

    specs = _specs(23, seed=7 + C)
    b, ins, outs, exact, pitches = _run_batch(rs, specs, C, dt, aligned)
    assert b.info.use_tma == (1 if aligned else 0)
    b(ins, outs)
    torch.cuda.synchronize()
    for i, sp in enumerate(specs):
        got = outs[i].double().cpu().numpy()
        want = oracle.resample(exact[i], got.shape[0], got.shape[1], sp["kernel"], sp["boundary"],
                               param=sp["param"])
        assert np.abs(got - want).max() <= TOL[dt], (i, sp)
        # alone, through the plan path, on the kernel the batch ran it on (the
        # tile kernel, or a streaming kernel in its untuned form), same pitch
        path = rs.rs_batch_image_path(b.handle, i)
        flags = {0: rs.RS_FORCE_SIMT | rs.RS_NO_STREAM, 3: rs.RS_FORCE_STREAM | rs.RS_FORCE_SIMT,
                 5: rs.RS_FORCE_STREAM}[path]
        d = rs.make_desc(sp["in_h"], sp["in_w"], C, got.shape[0], got.shape[1], kernel=sp["kernel"],
                         param=sp["param"], boundary=sp["boundary"], dtype=ins[i].dtype,
                         in_row_stride=pitches[i], flags=flags)
        h = rs.rs_plan_create(d, 0)
        alone = torch.empty_like(outs[i])
        rs.rs_resample(h, ins[i].data_ptr(), alone.data_ptr(), 0)
        torch.cuda.synchronize()
        rs.rs_destroy(h)
        assert torch.equal(alone, outs[i]), i
    with pytest.raises(rs.RSError) as e:
        rs.rs_batch_image_path(b.handle, len(specs))
    assert e.value.status == rs.RS_ERR_INVALID_ARG
    # replay with other output buffers (the graph re-stages the pointers)
    outs2 = [torch.zeros_like(o) for o in outs]
    b(ins, outs2)
    b(ins, outs)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    b.close()


def test_batch_autotune_keeps_results(rs, tmp_path):
    import torch

    specs = _specs(16, seed=3, side=(40, 400))
    b, ins, outs, exact, pitches = _run_batch(rs, specs, 1, "f16", True)
    b(ins, outs)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    cache = str(tmp_path / "batch.jsonl")
    b.autotune(ins, outs, cache_path=cache)
    assert len(open(cache).read().splitlines()) == 1
    b(ins, outs)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    b.close()


def test_batch_rejects_mixed_channels(rs):
    d0 = rs.make_desc(10, 10, 1, 5, 5, kernel="cubic", boundary="clamp", dtype=rs.RS_F32)
    d1 = rs.make_desc(10, 10, 3, 5, 5, kernel="cubic", boundary="clamp", dtype=rs.RS_F32)
    with pytest.raises(rs.RSError) as ei:
        rs.rs_batch_create([d0, d1], 0)
    assert ei.value.status == rs.RS_ERR_UNSUPPORTED


def test_batch_streams_large_images(rs):
    """Images of >= 2^18 output pixels run on the row-streaming kernel (bit-identical
    to that kernel alone), the rest on the persistent tile kernel."""
    import torch

    specs = [dict(in_h=800, in_w=824, scale=1.37, kernel="lanczos", param=3.0, boundary="mirror"),
             dict(in_h=120, in_w=96, scale=2.0, kernel="cubic", param=-0.5, boundary="clamp"),
             dict(in_h=700, in_w=720, scale=1.6, kernel="linear", param=None, boundary="reflect101"),
             dict(in_h=300, in_w=256, scale=0.5, kernel="lanczos", param=3.0, boundary="mirror")]
    b, ins, outs, exact, pitches = _run_batch(rs, specs, 1, "f16", True)
    big = [out.shape[0] * out.shape[1] >= (1 << 18) for out in outs]
    assert big == [True, False, True, False]
    assert b.info.n_streamed == 2
    b(ins, outs)
    torch.cuda.synchronize()
    g = np.random.default_rng(3)
    for i, sp in enumerate(specs):
        got = outs[i].double().cpu().numpy()
        rows = sorted(set([0, got.shape[0] - 1]) | set(int(r) for r in g.integers(0, got.shape[0], 6)))
        for r in rows:
            want = oracle.resample(exact[i], got.shape[0], got.shape[1], sp["kernel"], sp["boundary"],
                                   param=sp["param"], rows=(r, r + 1))[0]
            assert np.abs(got[r] - want).max() <= TOL["f16"], (i, r)
        flags = rs.RS_FORCE_STREAM if big[i] else rs.RS_FORCE_SIMT | rs.RS_NO_STREAM
        d = rs.make_desc(sp["in_h"], sp["in_w"], 1, got.shape[0], got.shape[1], kernel=sp["kernel"],
                         param=sp["param"], boundary=sp["boundary"], dtype=ins[i].dtype,
                         in_row_stride=pitches[i], flags=flags)
        h = rs.rs_plan_create(d, 0)
        assert rs.rs_plan_get_info(h).path == (3 if big[i] else 0)
        alone = torch.empty_like(outs[i])
        rs.rs_resample(h, ins[i].data_ptr(), alone.data_ptr(), 0)
        torch.cuda.synchronize()
        rs.rs_destroy(h)
        assert torch.equal(alone, outs[i]), i
    b.close()


def test_batch_band_images_share_one_launch(rs):
    """Several large images on the band kernels (mild downscales and a 2-tap
    upscale) run in one multi-image launch, each re-planned for its share of
    the SMs: every result is bit-identical to its band kernel alone, and
    within tolerance of the oracle on sampled rows."""
    import torch

    specs = [dict(in_h=1400, in_w=1400, scale=0.8, kernel="lanczos", param=3.0, boundary="mirror"),
             dict(in_h=1600, in_w=1600, scale=0.7, kernel="cubic", param=-0.5, boundary="clamp"),
             dict(in_h=700, in_w=720, scale=1.6, kernel="linear", param=None, boundary="reflect101"),
             dict(in_h=1200, in_w=1104, scale=0.9, kernel="lanczos", param=3.0, boundary="truncate"),
             dict(in_h=100, in_w=120, scale=0.6, kernel="cubic", param=-0.5, boundary="mirror")]
    b, ins, outs, exact, pitches = _run_batch(rs, specs, 1, "f16", True)
    big = [out.shape[0] * out.shape[1] >= (1 << 18) for out in outs]
    assert big == [True, True, True, True, False]
    assert b.info.n_streamed == 4
    b(ins, outs)
    torch.cuda.synchronize()
    g = np.random.default_rng(11)
    for i, sp in enumerate(specs):
        assert rs.rs_batch_image_path(b.handle, i) == (3 if big[i] else 0), i
        got = outs[i].double().cpu().numpy()
        rows = sorted(set([0, got.shape[0] - 1]) | set(int(r) for r in g.integers(0, got.shape[0], 4)))
        for r in rows:
            want = oracle.resample(exact[i], got.shape[0], got.shape[1], sp["kernel"], sp["boundary"],
                                   param=sp["param"], rows=(r, r + 1))[0]
            assert np.abs(got[r] - want).max() <= TOL["f16"], (i, r)
        flags = rs.RS_FORCE_STREAM | rs.RS_FORCE_SIMT if big[i] else rs.RS_FORCE_SIMT | rs.RS_NO_STREAM
        d = rs.make_desc(sp["in_h"], sp["in_w"], 1, got.shape[0], got.shape[1], kernel=sp["kernel"],
                         param=sp["param"], boundary=sp["boundary"], dtype=ins[i].dtype,
                         in_row_stride=pitches[i], flags=flags)
        h = rs.rs_plan_create(d, 0)
        assert rs.rs_plan_get_info(h).path == (3 if big[i] else 0)
        alone = torch.empty_like(outs[i])
        rs.rs_resample(h, ins[i].data_ptr(), alone.data_ptr(), 0)
        torch.cuda.synchronize()
        rs.rs_destroy(h)
        assert torch.equal(alone, outs[i]), i
    # a second run, on other output buffers (re-staged pointers), gives the same results
    outs2 = [torch.zeros_like(o) for o in outs]
    b(ins, outs2)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    b.close()
