"""rs_resample_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (a plug-in whose host application owns the device
memory, a real-time loop that may not pay for cudaMalloc/cudaFree).

Checked through the C ABI on calls in a row with different geometries (so
that whatever one call left in the shared static scratch cannot leak into the
next result): against the regular entry point (rs_plan_create + rs_resample)
within the tolerances the other tests use, bit for bit against a plan forced
onto the same two-pass kernels, and against the FP64 oracle; on FP32, FP64,
FP16 and BF16, packed and padded row strides.  It allocates nothing on a call
once its array exists (free device memory unchanged), rejects what it cannot
do with a clear status, and answers RS_ERR_BUDGET beyond its array.  This
file is named so that pytest collects it last.
"""
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


def _tdt(dt):
    import torch

    return {"f32": torch.float32, "f64": torch.float64, "f16": torch.float16, "bf16": torch.bfloat16}[dt]


def _plan_path(rs, desc, x, out_shape, flags=0):
    """The regular entry point on the same descriptor (optionally with extra
    plan flags), into a fresh output of the given (rows, row pitch) shape."""
    import torch

    d = rs.make_desc(desc.in_h, desc.in_w, desc.channels, desc.out_h, desc.out_w,
                     kernel=_KNAMES[desc.kernel], param=desc.param, boundary=_BNAMES[desc.boundary],
                     dtype=desc.in_dtype, flags=desc.flags | flags, in_row_stride=desc.in_row_stride,
                     out_row_stride=desc.out_row_stride)
    h = rs.rs_plan_create(d, 0)
    y = torch.full(out_shape, float("nan"), dtype=x.dtype, device="cuda")
    rs.rs_resample(h, x.data_ptr(), y.data_ptr(), 0)
    torch.cuda.synchronize()
    rs.rs_plan_check(h)
    rs.rs_destroy(h)
    return y


def _names(rs):
    global _KNAMES, _BNAMES
    _KNAMES = {v: k for k, v in rs.KERNELS.items()}
    _BNAMES = {v: k for k, v in rs.BOUNDARIES.items()}


# (in_h, in_w, C, out_h, out_w, kernel, boundary, dtype, input pitch pad, output pitch pad)
CASES = [
    (300, 420, 3, 411, 575, "lanczos", "mirror", "f32", 0, 0),     # x1.37
    (640, 480, 1, 192, 144, "lanczos", "mirror", "f32", 0, 0),     # x0.3, antialiased
    (256, 256, 1, 512, 512, "cubic", "clamp", "f64", 0, 0),        # x2 Keys, FP64
    (200, 333, 3, 61, 101, "linear", "truncate", "bf16", 0, 0),
    (150, 212, 3, 205, 290, "mitchell", "reflect101", "f16", 0, 0),
    (97, 130, 3, 131, 175, "lanczos", "mirror", "f32", 13, 7),     # padded row strides
]


def _run_case(rs, case):
    """(the entry point's result, the plan path's, the two-pass plan's, the
    oracle's) on the valid samples, as float64 numpy arrays."""
    import torch

    H, W, C, OH, OW, k, b, dt, pin, pout = case
    img = synth.sinusoids(H, W, C, seed=H * 7 + W)
    t = torch.from_numpy(img).to(_tdt(dt))
    exact = t.to(torch.float64).numpy()
    in_pitch, out_pitch = W * C + pin, OW * C + pout
    src = torch.zeros((H, in_pitch), dtype=_tdt(dt))
    src[:, :W * C] = t.reshape(H, W * C)
    x = src.cuda().contiguous()
    desc = rs.make_desc(H, W, C, OH, OW, kernel=k, boundary=b, dtype=_tdt(dt),
                        in_row_stride=in_pitch if pin else 0, out_row_stride=out_pitch if pout else 0)
    got = torch.full((OH, out_pitch), float("nan"), dtype=_tdt(dt), device="cuda")
    rs.rs_resample_noalloc(desc, x.data_ptr(), got.data_ptr(), 0)
    torch.cuda.synchronize()
    plan = _plan_path(rs, desc, x, (OH, out_pitch))
    two_pass = _plan_path(rs, desc, x, (OH, out_pitch), flags=rs.RS_TWO_PASS)
    want = oracle.resample(exact, OH, OW, k, b, param=desc.param)

    def valid(y):
        return y[:, :OW * C].double().cpu().numpy().reshape(OH, OW, C)

    return valid(got), valid(plan), valid(two_pass), want, got


def test_noalloc_matches_the_plan_path_twice_in_a_row(rs):
    _names(rs)
    for first, second in ((CASES[0], CASES[1]), (CASES[2], CASES[3]), (CASES[4], CASES[5])):
        for case in (first, second):
            dt = case[7]
            got, plan, two_pass, want, raw = _run_case(rs, case)
            assert np.isfinite(got).all(), case
            assert np.abs(got - plan).max() <= TOL[dt], case
            # the same kernels as a plan forced onto the two-pass path: bit for bit
            assert np.array_equal(got, two_pass), (case, np.abs(got - two_pass).max())
            assert np.abs(got - want).max() <= TOL[dt], (case, np.abs(got - want).max())
            if case[9]:
                # the padding after each output row is left untouched
                assert torch_isnan_all(raw[:, case[4] * case[2]:])


def torch_isnan_all(t):
    import torch

    return bool(torch.isnan(t.float()).all().item())


def test_noalloc_allocates_nothing_once_its_array_exists(rs):
    import torch

    _names(rs)
    H, W, C = 240, 320, 3
    x = torch.from_numpy(synth.sinusoids(H, W, C, seed=3)).cuda()
    desc = rs.make_desc(H, W, C, 329, 438, kernel="lanczos", boundary="mirror", dtype=torch.float32)
    y = torch.empty((329, 438, C), dtype=torch.float32, device="cuda")
    rs.rs_resample_noalloc(desc, x.data_ptr(), y.data_ptr(), 0)   # creates the array (lazy loading)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rs.rs_resample_noalloc(desc, x.data_ptr(), y.data_ptr(), 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_refuses_what_it_cannot_do(rs):
    import torch

    x = torch.empty(16, device="cuda")
    base = dict(kernel="lanczos", boundary="mirror", dtype=torch.float32)
    with pytest.raises(rs.RSError) as ei:          # the only flag it takes is RS_NO_ANTIALIAS
        rs.rs_resample_noalloc(rs.make_desc(64, 64, 1, 80, 80, flags=rs.RS_FORCE_STREAM, **base),
                               x.data_ptr(), x.data_ptr(), 0)
    assert ei.value.status == rs.RS_ERR_UNSUPPORTED
    with pytest.raises(rs.RSError) as ei:          # the same descriptor checks as rs_plan_create
        rs.rs_resample_noalloc(rs.make_desc(64, 64, 1, 80, 80, kernel="cubic", param=float("nan"),
                                            boundary="clamp", dtype=torch.float32),
                               x.data_ptr(), x.data_ptr(), 0)
    assert ei.value.status == rs.RS_ERR_INVALID_ARG and "cubic a" in rs.rs_last_error()
    desc = rs.make_desc(4096, 4096, 3, 5612, 5612, **base)
    with pytest.raises(rs.RSError) as ei:          # beyond the static array
        rs.rs_resample_noalloc(desc, x.data_ptr(), x.data_ptr(), 0)
    assert ei.value.status == rs.RS_ERR_BUDGET
    assert "static scratch" in rs.rs_last_error()
