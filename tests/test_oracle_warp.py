"""Pins of the EWA warp oracle (CPU): a uniform image stays uniform; an
identity warp is the Gaussian filter of width sigma sqrt(2) (scipy's
gaussian_filter, which samples the same Gaussian at the same offsets); a
quarter turn of a square image is the quarter-turned identity result; an
integer translation shifts it; the footprint widens with minification."""
import math

import numpy as np
import pytest
import scipy.ndimage as nd

from oracle import warp as ow


@pytest.mark.parametrize("boundary", ["clamp", "mirror", "reflect101"])
def test_uniform_stays_uniform(boundary):
    img = np.full((12, 15, 2), 0.42)
    for a in ((1, 0, 0, 0, 1, 0), (0.4, 0.1, 2.0, -0.2, 0.5, 1.0), (2.5, 0.0, -3.0, 0.0, 1.7, 0.5)):
        out = ow.warp(img, 9, 11, a, 0.5, 3.0, boundary)
        assert np.abs(out - 0.42).max() < 1e-14, (a, boundary)


@pytest.mark.parametrize("boundary,mode", [("clamp", "nearest"), ("mirror", "reflect"), ("reflect101", "mirror")])
@pytest.mark.parametrize("sigma", [0.5, 0.9])
def test_identity_is_a_gaussian_filter(boundary, mode, sigma):
    img = np.random.default_rng(1).random((17, 21))
    out = ow.warp(img, 17, 21, (1, 0, 0, 0, 1, 0), sigma, 8.0, boundary)
    ref = nd.gaussian_filter(img, sigma * math.sqrt(2.0), mode=mode, truncate=8.0)
    assert np.abs(out - ref).max() < 1e-12


def test_quarter_turn_and_translation():
    n = 14
    img = np.random.default_rng(2).random((n, n))
    base = ow.warp(img, n, n, (1, 0, 0, 0, 1, 0), 0.6, 3.0, "clamp")
    turned = ow.warp(img, n, n, (0, -1, n, 1, 0, 0), 0.6, 3.0, "clamp")
    assert np.abs(turned - np.rot90(base)).max() < 1e-13
    shifted = ow.warp(img, n, n, (1, 0, 3, 0, 1, -2), 0.6, 3.0, "clamp")
    assert np.abs(shifted[2:, :n - 3] - base[:n - 2, 3:]).max() < 1e-13


def test_footprint_widens_with_minification():
    V1 = ow.covariance((1, 0, 0, 0, 1, 0), 0.5)
    V4 = ow.covariance((4, 0, 0, 0, 0.5, 0), 0.5)
    assert np.allclose(V1, 0.5 * np.eye(2))
    assert np.allclose(V4, 0.25 * np.diag([17.0, 1.25]))
