"""Pins of the clustering oracle (CPU): the vectorised rounds against an
independent loop-by-loop brute force on tiny grids, and properties the
method fixes -- the merged region keeps the greater ID (so a region's ID is
its largest pixel index), the region count falls every round, the final
partition leaves no neighbouring pair within the thresholds (Eq. 1), region
descriptors are the means over their pixels, and closed special cases."""
import math

import numpy as np
import pytest

import synth
from oracle import cluster as oc


def _tiny(seed, h, w, levels=3):
    g = np.random.default_rng(seed)
    z = (1.0 + 0.05 * g.integers(0, levels, (h, w)) + g.normal(0, 0.01, (h, w))).astype(np.float32)
    d = (z * 1.1).astype(np.float32)
    inten = (g.uniform(0.2, 0.25, (h, w)) / (d.astype(np.float64) ** 2)).astype(np.float32)
    return z, d, inten


@pytest.mark.parametrize("seed", range(24))
def test_rounds_match_brute_force(seed):
    g = np.random.default_rng(100 + seed)
    h, w = int(g.integers(1, 8)), int(g.integers(1, 8))
    z, d, inten = _tiny(seed, h, w)
    for t_phi in (0.05, 0.009):
        L1, r1, *_ = oc.cluster(z, d, inten, t_phi=t_phi)
        L2, r2 = oc.brute(z, d, inten, t_phi=t_phi)
        assert np.array_equal(L1, L2) and r1 == r2, (h, w, t_phi)


def _qualifying_pairs(labels, mz, mp, t_z, t_phi):
    h, w = labels.shape
    bad = 0
    for y in range(h):
        for x in range(w):
            for yy, xx in ((y + 1, x), (y, x + 1)):
                if yy < h and xx < w:
                    R, S = labels[y, x], labels[yy, xx]
                    if R != S and abs(np.float32(mz[R] - mz[S])) <= t_z and abs(np.float32(mp[R] - mp[S])) <= t_phi:
                        bad += 1
    return bad


def test_invariants_on_a_synthetic_crop():
    Z, D, I = synth.tof_frames(1, 64, 72, seed=5)
    z, d, inten = Z[0], D[0], I[0]
    labels, rounds, counts, mz, mp, size = oc.cluster(z, d, inten)
    n = z.size
    assert rounds >= 1 and counts[0] == n
    assert all(b < a for a, b in zip(counts, counts[1:]))          # every round merges
    assert size.sum() == n and np.count_nonzero(size) == counts[-1]
    flat = labels.ravel()
    ph = oc.phi(d, inten).ravel().astype(np.float64)
    for R in np.unique(flat):
        pix = np.flatnonzero(flat == R)
        assert R == pix.max()                                        # greater ID kept
        assert size[R] == pix.size
        assert abs(mz[R] - z.ravel()[pix].astype(np.float64).mean()) < 1e-5 * max(1.0, abs(mz[R]))
        assert abs(mp[R] - ph[pix].mean()) < 1e-5
    assert _qualifying_pairs(labels, mz, mp, oc.T_Z, oc.T_PHI) == 0  # stopping rule


def test_special_cases():
    h, w = 9, 11
    one = np.ones((h, w), np.float32)
    # a uniform frame ends as one region carrying the largest pixel index
    labels, rounds, counts, *_ = oc.cluster(one, one, one)
    assert (labels == h * w - 1).all() and counts[-1] == 1
    # distinct values and zero thresholds: nothing merges
    g = np.random.default_rng(1)
    z = g.permutation(h * w).astype(np.float32).reshape(h, w)
    labels, rounds, counts, *_ = oc.cluster(z, one, one, t_z=0.0, t_phi=0.0)
    assert rounds == 0 and (labels == np.arange(h * w).reshape(h, w)).all()
    # two flat surfaces 0.5 m apart: exactly two regions, split where they meet
    z = np.where(np.arange(w)[None, :] < 4, 1.0, 1.5).astype(np.float32) * one
    labels, *_ = oc.cluster(z, z, 1.0 / (z * z))
    assert (labels[:, :4] == (h - 1) * w + 3).all() and (labels[:, 4:] == h * w - 1).all()


def test_phi_closed_forms():
    # d sqrt(I) = 1: arctan 1 = pi / 4; d sqrt(I) = sqrt(3): pi / 3
    assert oc.phi(np.float32(2.0), np.float32(0.25)) == np.float32(math.pi / 4)
    assert oc.phi(np.float32(1.0), np.float32(3.0)) == np.float32(math.atan(math.sqrt(np.float32(3.0))))
    assert oc.phi(np.float32(0.0), np.float32(5.0)) == 0.0


def test_paper_constants():
    """Table 1: t_z = 0.04 m, t_phi = 0.009 rad, alpha_z = 8 / pi, alpha_phi = 4 / 3."""
    assert oc.T_Z == np.float32(0.04) and oc.T_PHI == np.float32(0.009)
    assert oc.ALPHA_Z == np.float32(8 / math.pi) and oc.ALPHA_PHI == np.float32(4 / 3)
