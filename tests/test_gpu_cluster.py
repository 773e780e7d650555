"""The clustering kernel (the paper's parallel merging) against the CPU
oracle: partitions, region IDs, round counts and region descriptors are
bit-exact (both take every decision in FP32 with the same rounding), on tiny
random grids, synthetic ToF frames batched in one launch, full 204 x 204
frames, a round cap and the degenerate cases."""
import numpy as np
import pytest

import synth
from oracle import cluster as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_5450_b300 as rs

    return rs


def _run(rs, Z, D, I, regions=True, **kw):
    import torch

    n, h, w = Z.shape
    c = rs.Cluster(n, h, w, **kw)
    out = c(*(torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in (Z, D, I)), regions=regions)
    torch.cuda.synchronize()
    c.close()
    return [t.cpu().numpy() for t in out]


def _check_frame(lab, rnd, rz, rp, rn, z, d, inten, **kw):
    want_lab, want_rounds, _, mz, mp, size = oc.cluster(z, d, inten, **kw)
    assert rnd == want_rounds
    assert np.array_equal(lab, want_lab)
    assert np.array_equal(rn.ravel(), size.astype(np.int32))
    live = size > 0
    assert np.array_equal(rz.ravel()[live], mz[live]) and np.array_equal(rp.ravel()[live], mp[live])


def _tiny(seed, h, w):
    g = np.random.default_rng(seed)
    z = (1.0 + 0.05 * g.integers(0, 3, (h, w)) + g.normal(0, 0.01, (h, w))).astype(np.float32)
    d = (z * 1.1).astype(np.float32)
    inten = (g.uniform(0.2, 0.25, (h, w)) / (d.astype(np.float64) ** 2)).astype(np.float32)
    return z, d, inten


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (7, 1), (5, 6), (13, 17)])
def test_tiny_grids(rs, seed, shape):
    h, w = shape
    z, d, inten = _tiny(seed, h, w)
    for t_phi in (0.05, 0.009):
        lab, rnd, rz, rp, rn = _run(rs, z[None], d[None], inten[None], t_phi=t_phi)
        _check_frame(lab[0], rnd[0], rz[0], rp[0], rn[0], z, d, inten, t_phi=t_phi)


def test_batched_synthetic_frames(rs):
    Z, D, I = synth.tof_frames(6, 64, 72, seed=3)
    lab, rnd, rz, rp, rn = _run(rs, Z, D, I)
    for k in range(6):
        _check_frame(lab[k], rnd[k], rz[k], rp[k], rn[k], Z[k], D[k], I[k])


def test_full_frames(rs):
    Z, D, I = synth.tof_frames(2)
    lab, rnd, rz, rp, rn = _run(rs, Z, D, I)
    for k in range(2):
        _check_frame(lab[k], rnd[k], rz[k], rp[k], rn[k], Z[k], D[k], I[k])


def test_round_cap(rs):
    Z, D, I = synth.tof_frames(1, 40, 40, seed=9)
    lab, rnd, rz, rp, rn = _run(rs, Z, D, I, max_rounds=3)
    assert rnd[0] == 3
    _check_frame(lab[0], rnd[0], rz[0], rp[0], rn[0], Z[0], D[0], I[0], max_rounds=3)


def test_degenerate_cases(rs):
    h, w = 9, 11
    one = np.ones((1, h, w), np.float32)
    lab, rnd, *_ = _run(rs, one, one, one)
    assert (lab == h * w - 1).all()
    # zero thresholds and distinct depths: no merge, and the region phi is each
    # pixel's phi = arctan(d sqrt(I))
    g = np.random.default_rng(2)
    z = g.permutation(h * w).astype(np.float32).reshape(1, h, w)
    d = g.uniform(0.5, 3.0, (1, h, w)).astype(np.float32)
    inten = g.uniform(0.01, 1.0, (1, h, w)).astype(np.float32)
    lab, rnd, rz, rp, rn = _run(rs, z, d, inten, t_z=0.0, t_phi=0.0)
    assert rnd[0] == 0 and (lab[0] == np.arange(h * w).reshape(h, w)).all()
    assert np.array_equal(rp[0].reshape(h, w), oc.phi(d[0], inten[0]))


def test_rejects_bad_descriptors(rs):
    for kw in (dict(t_z=-1.0), dict(alpha_phi=float("inf")), dict(max_rounds=-2)):
        with pytest.raises(RuntimeError):
            rs.Cluster(1, 8, 8, **kw)
    with pytest.raises(RuntimeError):
        rs.Cluster(1, 1 << 13, 1 << 12)
