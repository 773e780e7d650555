"""rs_resample_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (a plug-in whose host application owns the device
memory, a real-time loop that may not pay for cudaMalloc/cudaFree).

It is checked through the C ABI against the regular plan path
(rs_plan_create + rs_resample) on two calls in a row, the second with a
different geometry so that whatever the first call left in the shared static
scratch cannot leak into the result.  This file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

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


def _plan_path(rs, desc, x):
    import torch

    h = rs.rs_plan_create(desc, 0)
    info = rs.rs_plan_get_info(h)
    y = torch.empty((info.out_h, info.out_w, desc.channels), dtype=x.dtype, device="cuda")
    rs.rs_resample(h, x.data_ptr(), y.data_ptr(), 0)
    torch.cuda.synchronize()
    rs.rs_plan_check(h)
    rs.rs_destroy(h)
    return y


CASES = [
    # (in_h, in_w, C, out_h, out_w, kernel, boundary, dtype)
    (300, 420, 3, 411, 575, "lanczos", "mirror", "f32"),   # x1.37
    (640, 480, 1, 192, 144, "lanczos", "mirror", "f32"),   # x0.3, antialiased
    (256, 256, 1, 512, 512, "cubic", "clamp", "f64"),      # x2 Keys, FP64
    (200, 333, 3, 61, 101, "linear", "truncate", "bf16"),
]


def test_noalloc_matches_plan_path_twice_in_a_row(rs):
    import torch

    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}
    for first, second in ((CASES[0], CASES[1]), (CASES[2], CASES[3])):
        for (H, W, C, OH, OW, k, b, dt) in (first, second):
            img = synth.sinusoids(H, W, C, seed=H * 7 + W)
            x = torch.from_numpy(img).to(tdt[dt]).cuda().contiguous()
            desc = rs.make_desc(H, W, C, OH, OW, kernel=k, boundary=b, dtype=tdt[dt])
            want = _plan_path(rs, desc, x)
            got = torch.full_like(want, float("nan"))
            rs.rs_resample_noalloc(desc, x.data_ptr(), got.data_ptr(), 0)
            torch.cuda.synchronize()
            err = (got.double() - want.double()).abs().max().item()
            assert np.isfinite(err) and err <= TOL[dt], (H, W, OH, OW, k, b, dt, err)


def test_noalloc_rejects_requests_beyond_the_static_scratch(rs):
    import torch

    desc = rs.make_desc(4096, 4096, 3, 5612, 5612, kernel="lanczos", boundary="mirror",
                        dtype=torch.float32)
    x = torch.empty(1, device="cuda")
    with pytest.raises(rs.RSError) as ei:
        rs.rs_resample_noalloc(desc, x.data_ptr(), x.data_ptr(), 0)
    assert ei.value.status == rs.RS_ERR_BUDGET
    assert "static scratch" in rs.rs_last_error()
