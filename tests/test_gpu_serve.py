"""Serving: continuous batching under a memory budget.  Every request's
result is compared with the FP64 oracle and, bit for bit, with the same
resample run alone through the plan path."""
import time

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


def _base(rs, side, C, dt, seed):
    """A padded device image (16-byte row pitch) and its exact float64 copy."""
    import torch

    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dt]
    img = synth.sinusoids(side, side, C, seed=seed)
    t = torch.from_numpy(img).to(tdt)
    vec = 16 // t.element_size()
    row = side * C
    pitch = (row + vec - 1) // vec * vec
    buf = torch.zeros((side, pitch), dtype=tdt, device="cuda")
    buf[:, :row] = t.reshape(side, row).cuda()
    return buf, t.double().numpy(), pitch


def _wait(rs, srv, tickets, timeout=60.0):
    t0 = time.time()
    states = {}
    while len(states) < len(tickets):
        for tk in tickets:
            if tk in states:
                continue
            st = rs.rs_batch_poll(srv, tk)
            if st.status != rs.RS_ERR_BUSY:
                states[tk] = st
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.001)
    return states


def _alone(rs, desc, d_in, out_shape, tdt):
    import torch

    h = rs.rs_plan_create(desc, 0)
    y = torch.empty(out_shape, dtype=tdt, device="cuda")
    rs.rs_resample(h, d_in, y.data_ptr(), 0)
    torch.cuda.synchronize()
    rs.rs_destroy(h)
    return y


class _DevicePtr:
    """A raw device pointer exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3}


def _view(rs, st, C, tdt):
    """Copy of a server-owned output as a (out_h, out_w, C) tensor."""
    import torch

    es = torch.empty((), dtype=tdt).element_size()
    raw = torch.as_tensor(_DevicePtr(st.d_out, st.out_h * st.out_row_stride * es), device="cuda")
    rows = raw.view(tdt).reshape(st.out_h, st.out_row_stride)[:, :st.out_w * C]
    return rows.reshape(st.out_h, st.out_w, C).clone()


CASES = [  # (side, C, dtype, scale, kernel, param)
    (97, 3, "bf16", 1.9, "cubic", -0.5), (200, 1, "bf16", 0.3, "lanczos", 3.0), (64, 3, "f16", 4.0, "lanczos", 3.0),
    (333, 1, "f16", 0.125, "cubic", -0.5), (120, 3, "f32", 1.37, "lanczos", 3.0), (45, 1, "f32", 2.5, "linear", None),
    (150, 3, "bf16", 0.61, "lanczos", 3.0), (77, 1, "bf16", 7.3, "cubic", -0.5),
]


def test_server_results_match_oracle_and_alone(rs):
    import torch

    tdts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    srv = rs.rs_server_create(2 << 30, max_inflight=3, max_batch=4)
    bases = {}
    reqs, meta = [], []
    for k, (side, C, dt, scale, kern, par) in enumerate(CASES * 3):
        key = (side, C, dt)
        if key not in bases:
            bases[key] = _base(rs, side, C, dt, seed=side + C)
        buf, exact, pitch = bases[key]
        desc = rs.make_desc(side, side, C, scale_h=scale, scale_w=scale, kernel=kern, param=par,
                            boundary="mirror", dtype=tdts[dt], in_row_stride=pitch)
        reqs.append(rs.rs_request(desc, buf.data_ptr(), None))
        meta.append((key, scale, kern, par, dt, C))
    # two waves: the second arrives while the first is running
    t1 = rs.rs_batch_submit(srv, reqs[:12])
    t2 = rs.rs_batch_submit(srv, reqs[12:])
    tickets = list(range(t1, t1 + 12)) + list(range(t2, t2 + len(reqs) - 12))
    states = _wait(rs, srv, tickets)
    rs.rs_server_drain(srv)
    for tk, (key, scale, kern, par, dt, C) in zip(tickets, meta):
        st = states[tk]
        assert st.status == rs.RS_OK, (tk, st.status)
        buf, exact, pitch = bases[key]
        got = _view(rs, st, C, tdts[dt])
        want = oracle.resample(exact, st.out_h, st.out_w, kern, "mirror", param=par)
        assert np.abs(got.double().cpu().numpy() - want).max() <= TOL[dt], (tk, key, scale)
        # the server runs the SIMT kernel: compare with a plan kept off the tensor cores
        desc = rs.make_desc(key[0], key[0], C, st.out_h, st.out_w, kernel=kern, param=par, boundary="mirror",
                            dtype=tdts[dt], in_row_stride=pitch, flags=rs.RS_FORCE_SIMT | rs.RS_NO_STREAM)
        alone = _alone(rs, desc, buf.data_ptr(), (st.out_h, st.out_w, C), tdts[dt])
        assert torch.equal(alone, got), (tk, key, scale)
        rs.rs_server_release(srv, tk)
    stats = rs.rs_server_get_stats(srv)
    assert stats.completed == len(reqs) and stats.rejected == 0
    assert stats.launches >= 3 and stats.max_batch <= 4
    assert stats.bytes_in_use == 0
    rs.rs_server_destroy(srv)


def test_server_budget_admission(rs):
    import torch

    buf, exact, pitch = _base(rs, 256, 1, "bf16", seed=5)
    # each request's output is 512*512*2 = 512 KiB (+ tables); the budget holds only a few
    srv = rs.rs_server_create(3 << 20, max_inflight=2, max_batch=8)
    desc = rs.make_desc(256, 256, 1, 512, 512, kernel="cubic", param=-0.5, boundary="clamp",
                        dtype=torch.bfloat16, in_row_stride=pitch)
    t = rs.rs_batch_submit(srv, [rs.rs_request(desc, buf.data_ptr(), None)] * 12)
    tickets = list(range(t, t + 12))
    done = []
    t0 = time.time()
    while len(done) < 12:
        for tk in tickets:
            if tk in done:
                continue
            st = rs.rs_batch_poll(srv, tk)
            if st.status == rs.RS_OK:
                done.append(tk)
                rs.rs_server_release(srv, tk)  # frees its output, letting the next ones in
        assert time.time() - t0 < 60
        time.sleep(0.001)
    stats = rs.rs_server_get_stats(srv)
    assert stats.max_bytes_in_use <= 3 << 20
    # a request that can never fit
    big = rs.make_desc(256, 256, 1, 4096, 4096, kernel="cubic", param=-0.5, boundary="clamp",
                       dtype=torch.bfloat16, in_row_stride=pitch)
    tb = rs.rs_batch_submit(srv, [rs.rs_request(big, buf.data_ptr(), None)])
    st = _wait(rs, srv, [tb])[tb]
    assert st.status == rs.RS_ERR_BUDGET
    rs.rs_server_destroy(srv)


def test_server_rejects_malformed_requests(rs):
    import torch

    buf, exact, pitch = _base(rs, 64, 1, "f32", seed=1)
    srv = rs.rs_server_create(64 << 20)
    bad = rs.make_desc(64, 64, 1, 32, 32, kernel="lanczos", param=3.0, boundary="mirror",
                       dtype=torch.float32, in_row_stride=pitch)
    bad.param = 2.5
    t = rs.rs_batch_submit(srv, [rs.rs_request(bad, buf.data_ptr(), None)])
    assert _wait(rs, srv, [t])[t].status == rs.RS_ERR_INVALID_ARG
    with pytest.raises(rs.RSError):
        rs.rs_batch_poll(srv, 999999)
    rs.rs_server_destroy(srv)


BIG_CASES = [  # (side, C, dtype, scale, kernel, param, boundary): at least 2^20 output pixels each
    (1024, 3, "f32", 1.37, "lanczos", 3.0, "mirror"),     # the pipelined kernel
    (800, 1, "bf16", 1.9, "cubic", -0.5, "clamp"),
    (1030, 3, "f32", 1.13, "cubic", -0.5, "reflect101"),
    (2048, 3, "f16", 0.6, "lanczos", 3.0, "mirror"),      # downscale: the band kernels
    (1500, 1, "bf16", 0.71, "lanczos", 2.0, "truncate"),
]


def _sample_rows(n, k, seed):
    g = np.random.default_rng(seed)
    rows = set([0, 1, n // 2, n - 2, n - 1]) | set(int(r) for r in g.integers(0, n, k))
    return sorted(r for r in rows if 0 <= r < n)


def test_server_large_requests_stream(rs):
    """Requests of 2^20 output pixels or more run alone on the row-streaming
    kernels, with window starts from the host's closed form: each result is
    bit-identical to a plan forced onto the streaming kernels (untuned, its
    starts read back from the device tables) and within tolerance of the
    oracle on sampled rows; small requests submitted beside them still batch."""
    import torch

    tdts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    srv = rs.rs_server_create(4 << 30, max_inflight=3, max_batch=8)
    reqs, meta = [], []
    for side, C, dt, scale, kern, par, bnd in BIG_CASES:
        buf, exact, pitch = _base(rs, side, C, dt, seed=side + 7 * C)
        desc = rs.make_desc(side, side, C, scale_h=scale, scale_w=scale, kernel=kern, param=par,
                            boundary=bnd, dtype=tdts[dt], in_row_stride=pitch)
        reqs.append(rs.rs_request(desc, buf.data_ptr(), None))
        meta.append((side, C, dt, kern, par, bnd, buf, exact, pitch))
    small, sexact, spitch = _base(rs, 97, 3, "bf16", seed=3)
    sdesc = rs.make_desc(97, 97, 3, scale_h=1.9, scale_w=1.9, kernel="cubic", param=-0.5, boundary="mirror",
                         dtype=torch.bfloat16, in_row_stride=spitch)
    reqs += [rs.rs_request(sdesc, small.data_ptr(), None)] * 4
    t0 = rs.rs_batch_submit(srv, reqs)
    tickets = list(range(t0, t0 + len(reqs)))
    states = _wait(rs, srv, tickets, timeout=120.0)
    rs.rs_server_drain(srv)
    for tk, (side, C, dt, kern, par, bnd, buf, exact, pitch) in zip(tickets, meta):
        st = states[tk]
        assert st.status == rs.RS_OK, (side, st.status)
        assert st.out_h * st.out_w >= 1 << 20 and st.batch_size == 1
        got = _view(rs, st, C, tdts[dt])
        desc = rs.make_desc(side, side, C, st.out_h, st.out_w, kernel=kern, param=par, boundary=bnd,
                            dtype=tdts[dt], in_row_stride=pitch, flags=rs.RS_FORCE_STREAM)
        alone = _alone(rs, desc, buf.data_ptr(), (st.out_h, st.out_w, C), tdts[dt])
        assert torch.equal(alone, got), (side, dt, bnd)
        err = 0.0
        for r in _sample_rows(st.out_h, 6, side):
            want = oracle.resample(exact, st.out_h, st.out_w, kern, bnd, param=par, rows=(r, r + 1))
            err = max(err, float(np.abs(got[r].double().cpu().numpy() - want[0]).max()))
        assert err <= TOL[dt], (side, dt, bnd, err)
        rs.rs_server_release(srv, tk)
    sts = [states[tk] for tk in tickets[len(BIG_CASES):]]
    assert all(s.status == rs.RS_OK for s in sts)
    ref = _view(rs, sts[0], 3, torch.bfloat16)
    for s in sts[1:]:
        assert torch.equal(_view(rs, s, 3, torch.bfloat16), ref)
    stats = rs.rs_server_get_stats(srv)
    assert stats.streamed == len(BIG_CASES), stats.streamed
    assert stats.launches <= len(BIG_CASES) + 4
    rs.rs_server_destroy(srv)


def test_server_launches_run_concurrently(rs):
    """Launches on different streams overlap on the device: the GPU-clock
    intervals (start and end of each launch's work) of two launches
    intersect.  Four classes (channels x dtype) give four launches per wave
    on four streams."""
    import torch

    tdts = {"f32": torch.float32, "bf16": torch.bfloat16}
    srv = rs.rs_server_create(2 << 30, max_inflight=4, max_batch=8)
    bases = {(C, dt): _base(rs, 720, C, dt, seed=11 + C) for C in (1, 3) for dt in ("f32", "bf16")}
    found = False
    for wave in range(4):
        reqs = []
        for (C, dt), (buf, exact, pitch) in bases.items():
            desc = rs.make_desc(720, 720, C, scale_h=1.4, scale_w=1.4, kernel="lanczos", param=3.0,
                                boundary="mirror", dtype=tdts[dt], in_row_stride=pitch)
            reqs += [rs.rs_request(desc, buf.data_ptr(), None)] * 2
        t0 = rs.rs_batch_submit(srv, reqs)
        tickets = list(range(t0, t0 + len(reqs)))
        states = _wait(rs, srv, tickets)
        spans = {}
        for tk in tickets:
            st = states[tk]
            assert st.status == rs.RS_OK
            assert 0 < st.t_gpu_start_ns < st.t_gpu_end_ns
            assert st.t_launch_ns <= st.t_done_ns
            if st.launch_id in spans:   # requests of one launch share its interval
                assert spans[st.launch_id] == (st.t_gpu_start_ns, st.t_gpu_end_ns)
            spans[st.launch_id] = (st.t_gpu_start_ns, st.t_gpu_end_ns)
            rs.rs_server_release(srv, tk)
        iv = sorted(spans.values())
        if any(b[0] < a[1] for a, b in zip(iv, iv[1:])):
            found = True
            break
    assert found, "no two launches overlapped on the device"
    rs.rs_server_destroy(srv)
