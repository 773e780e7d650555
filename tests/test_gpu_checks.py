"""Device-side checks and the failure path, without faulting or hanging a GPU.

* RS_CHECK: caller-supplied weights (rs_plan_set_weights) that are not finite
  or do not sum to one make the table check set the plan's error word, which
  rs_plan_check reports as RS_ERR_DEVICE; good custom weights pass the check
  and give the separable sum the tables define, on every kernel path.
* Bounded waits: rs_plan_wait_selftest runs the library's bounded mbarrier
  wait on a barrier nobody arrives on with a 1 ms limit; it gives up,
  rs_plan_check reports RS_ERR_TIMEOUT, and the plan resamples correctly
  afterwards (the context stays usable).
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


def _separable(img, start_y, wy, start_x, wx):
    """out[y][x][c] = sum_j sum_i wy[y][j] wx[x][i] img[start_y[y] + j][start_x[x] + i][c]."""
    H, W, C = img.shape
    ty, tx = wy.shape[1], wx.shape[1]
    rows = np.stack([img[start_y[y]:start_y[y] + ty] for y in range(len(start_y))])   # (OH, ty, W, C)
    tmp = np.einsum("yj,yjwc->ywc", wy, rows)                                            # (OH, W, C)
    cols = np.stack([tmp[:, start_x[x]:start_x[x] + tx] for x in range(len(start_x))], 1)  # (OH, OW, tx, C)
    return np.einsum("xi,yxic->yxc", wx, cols)


PATHS = [("default", 0), ("two_pass", 0x08), ("tiles", 0x20)]


@pytest.mark.parametrize("name,flags", PATHS, ids=[p[0] for p in PATHS])
def test_custom_weights_pass_the_check_and_are_applied(rs, name, flags):
    import torch

    H, W, C, OH, OW = 60, 84, 3, 83, 115
    img = synth.uniform(H, W, C, seed=41).astype(np.float32)
    x = torch.from_numpy(img).cuda()
    p = rs.Plan(H, W, C, OH, OW, kernel="lanczos", param=3.0, boundary="mirror", flags=flags | rs.RS_CHECK)
    tabs = [p.tables(a) for a in (0, 1)]
    g = np.random.default_rng(3)
    custom = []
    for a in (0, 1):
        w = tabs[a][4] + g.uniform(-0.05, 0.05, tabs[a][4].shape)
        w /= w.sum(1, keepdims=True)                       # still a partition of one
        rs.rs_plan_set_weights(p.handle, a, w, torch.cuda.current_stream().cuda_stream)
        custom.append(w)
    y = p(x)
    torch.cuda.synchronize()
    p.check()                                              # the check passes
    got = y.double().cpu().numpy()
    wy32, wx32 = custom[0].astype(np.float32).astype(np.float64), custom[1].astype(np.float32).astype(np.float64)
    want = _separable(img.astype(np.float64), tabs[0][2], wy32, tabs[1][2], wx32)
    assert np.abs(got - want).max() <= TOL["f32"], (name, p.path)
    # rs_plan_recompute restores the plan's own weights
    p.recompute()
    y = p(x)
    torch.cuda.synchronize()
    p.check()
    ref = oracle.resample(img.astype(np.float64), OH, OW, "lanczos", "mirror", param=3.0)
    assert np.abs(y.double().cpu().numpy() - ref).max() <= TOL["f32"]
    p.close()


@pytest.mark.parametrize("bad", ["nan", "sum"])
@pytest.mark.parametrize("name,flags", PATHS, ids=[p[0] for p in PATHS])
def test_rs_check_reports_bad_weights(rs, bad, name, flags):
    import torch

    H, W, C, OH, OW = 60, 84, 3, 83, 115
    x = torch.from_numpy(synth.uniform(H, W, C, seed=42).astype(np.float32)).cuda()
    p = rs.Plan(H, W, C, OH, OW, kernel="cubic", param=-0.5, boundary="clamp", flags=flags | rs.RS_CHECK)
    w = p.tables(1)[4].copy()
    if bad == "nan":
        w[17, 1] = np.nan
    else:
        w[17] *= 1.1                                       # sums to 1.1
    rs.rs_plan_set_weights(p.handle, 1, w, torch.cuda.current_stream().cuda_stream)
    p(x)
    torch.cuda.synchronize()
    with pytest.raises(rs.RSError) as ei:
        p.check()
    assert ei.value.status == rs.RS_ERR_DEVICE and "RS_CHECK" in rs.rs_last_error()
    # without RS_CHECK the same weights are used as given (no check, no error)
    q = rs.Plan(H, W, C, OH, OW, kernel="cubic", param=-0.5, boundary="clamp", flags=flags)
    rs.rs_plan_set_weights(q.handle, 1, w, torch.cuda.current_stream().cuda_stream)
    q(x)
    torch.cuda.synchronize()
    q.check()
    p.close()
    q.close()


def test_bounded_wait_runs_out_and_the_context_survives(rs):
    import time

    import torch

    H, W, C = 64, 96, 3
    img = synth.uniform(H, W, C, seed=43).astype(np.float32)
    x = torch.from_numpy(img).cuda()
    p = rs.Plan(H, W, C, 88, 131, kernel="lanczos", param=3.0, boundary="mirror")
    s = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    rs.rs_plan_wait_selftest(p.handle, 1000, s)            # 1 ms limit
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    with pytest.raises(rs.RSError) as ei:
        p.check()
    assert ei.value.status == rs.RS_ERR_TIMEOUT, rs.rs_last_error()
    assert waited < 1.0, waited                            # it gave up on its own limit
    p.check()                                              # the word was cleared
    y = p(x)                                               # and the context is usable
    torch.cuda.synchronize()
    p.check()
    want = oracle.resample(img.astype(np.float64), 88, 131, "lanczos", "mirror", param=3.0)
    assert np.abs(y.double().cpu().numpy() - want).max() <= TOL["f32"]
    with pytest.raises(rs.RSError) as ei:
        rs.rs_plan_wait_selftest(p.handle, 0, s)
    assert ei.value.status == rs.RS_ERR_INVALID_ARG
    p.close()
