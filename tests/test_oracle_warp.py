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


# ---------------------------------------------------------------------------
# The anisotropic part, against an independent construction of the filter.
#
# The EWA filter in input space is the reconstruction Gaussian (covariance
# sigma^2 I) convolved with the output-space prefilter (covariance sigma^2 I
# in output pixels) carried into the input by J: its density at offset d is
#     dens(d) = integral over u of  g(d - J u) g(u) du,  g(x) = exp(-|x|^2 / (2 sigma^2)),
# evaluated below by 2-D Gauss-Hermite quadrature in u, with no covariance
# matrix anywhere; Q(d) = -2 log(dens(d) / dens(0)) is then the quadratic
# form the oracle must reproduce (a Gaussian density is exp(-Q/2) times its
# value at 0).  The maps are non-normal (J J^T != J^T J) and have off-diagonal
# covariance, so a transposed product or a dropped cross term shows.

MAPS = [(1.0, 0.5, 0.3, 0.0, 1.0, -0.2),                      # shear
        (1.3856, -0.4, 0.1, 0.8, 0.6928, 0.4),               # rotation by 30 deg of a 1.6 x 0.8 scaling
        (0.9, 0.35, -0.5, -0.25, 1.2, 0.7)]                  # general


def _gh(n):
    t, w = np.polynomial.hermite.hermgauss(n)
    return t, w


def q_quadrature(a, sigma, d, n=72):
    """Q(d) for offsets d (..., 2) from the convolution integral (see above)."""
    J = np.array([[a[0], a[1]], [a[3], a[4]]], dtype=np.float64)
    t, w = _gh(n)
    u = math.sqrt(2.0) * sigma * np.stack(np.meshgrid(t, t, indexing="ij"), -1).reshape(-1, 2)  # (n^2, 2)
    wu = np.outer(w, w).reshape(-1)
    Ju = u @ J.T                                                                                # J u per node
    d = np.asarray(d, dtype=np.float64)
    diff = d[..., None, :] - Ju                                                                 # (..., n^2, 2)
    dens = (np.exp(-(diff ** 2).sum(-1) / (2.0 * sigma * sigma)) * wu).sum(-1)
    dens0 = (np.exp(-(Ju ** 2).sum(-1) / (2.0 * sigma * sigma)) * wu).sum(-1)
    return -2.0 * np.log(dens / dens0)


@pytest.mark.parametrize("a", MAPS)
@pytest.mark.parametrize("sigma", [0.5, 0.9])
def test_covariance_is_the_pushed_prefilter_plus_reconstruction(a, sigma):
    """V - sigma^2 I is the covariance of a sigma-wide output Gaussian pushed
    through J: its quadratic form at s is |J^-1 s|^2 / sigma^2 (solved, not
    formed from a product)."""
    J = np.array([[a[0], a[1]], [a[3], a[4]]])
    M = ow.covariance(a, sigma) - sigma * sigma * np.eye(2)
    s = np.random.default_rng(5).normal(size=(40, 2))
    lhs = np.einsum("ni,ij,nj->n", s, np.linalg.inv(M), s)
    rhs = (np.linalg.solve(J, s.T).T ** 2).sum(1) / (sigma * sigma)
    assert np.abs(lhs - rhs).max() < 1e-10 * rhs.max()


@pytest.mark.parametrize("a", MAPS)
def test_quadratic_form_matches_the_convolution_integral(a):
    sigma = 0.6
    g = np.random.default_rng(6)
    d = g.uniform(-2.5, 2.5, size=(200, 2))
    q = q_quadrature(a, sigma, d)
    Vi = np.linalg.inv(ow.covariance(a, sigma))
    q_or = np.einsum("ni,ij,nj->n", d, Vi, d)
    assert np.abs(q - q_or).max() < 1e-9 * max(1.0, q.max())
    # the quadrature has converged: more nodes give the same values
    assert np.abs(q - q_quadrature(a, sigma, d, n=96)).max() < 1e-11 * max(1.0, q.max())


def ewa_independent(img, out_h, out_w, a, sigma, cutoff):
    """The warp written from the definition with Q from the convolution
    integral (clamp boundary, one channel)."""
    H, W = img.shape
    r2 = cutoff * cutoff
    out = np.zeros((out_h, out_w))
    jj, ii = np.meshgrid(np.arange(-12, H + 12), np.arange(-12, W + 12), indexing="ij")
    js, is_ = jj.reshape(-1), ii.reshape(-1)
    vals = img[np.clip(js, 0, H - 1), np.clip(is_, 0, W - 1)]
    for y in range(out_h):
        for x in range(out_w):
            cu = a[0] * (x + 0.5) + a[1] * (y + 0.5) + a[2]
            cv = a[3] * (x + 0.5) + a[4] * (y + 0.5) + a[5]
            d = np.stack([is_ + 0.5 - cu, js + 0.5 - cv], -1)
            near = (np.abs(d) < 10.0).all(-1)  # the footprints here reach ~4 samples from the centre
            q = q_quadrature(a, sigma, d[near])
            w = np.where(q < r2, np.exp(-q / 2.0) - math.exp(-r2 / 2.0), 0.0)
            out[y, x] = (w * vals[near]).sum() / w.sum()
    return out


@pytest.mark.parametrize("a", MAPS[:2])
def test_anisotropic_warp_against_the_convolution_integral(a):
    """Whole warps with off-diagonal covariance and a small cutoff (r = 3, where
    the lowering by exp(-r^2/2) matters), oracle against the independent
    construction above."""
    img = np.random.default_rng(7).random((9, 11))
    out = ow.warp(img, 7, 8, a, 0.6, 3.0, "clamp")
    ref = ewa_independent(img, 7, 8, a, 0.6, 3.0)
    assert np.abs(out - ref).max() < 1e-9


# Planted mistakes in the warp oracle: each must fail one of the pins above.
WARP_MUTANTS = [
    ("jjt_transposed", "return (sigma * sigma) * (J @ J.T + np.eye(2))", "return (sigma * sigma) * (J.T @ J + np.eye(2))"),
    ("cross_term_dropped", "q = Vi[0, 0] * du * du + 2.0 * Vi[0, 1] * du * dv + Vi[1, 1] * dv * dv",
     "q = Vi[0, 0] * du * du + Vi[1, 1] * dv * dv"),
    ("cross_term_halved", "2.0 * Vi[0, 1] * du * dv", "Vi[0, 1] * du * dv"),
    ("no_lowering", "w = math.exp(-q / 2.0) - wcut", "w = math.exp(-q / 2.0)"),
    ("no_reconstruction_filter", "(J @ J.T + np.eye(2))", "(J @ J.T)"),
]


@pytest.mark.parametrize("name,old,new", WARP_MUTANTS, ids=[m[0] for m in WARP_MUTANTS])
def test_planted_warp_mistake_is_caught(name, old, new):
    import types

    src = open(ow.__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("warp_mutant_" + name)
    mod.__dict__["__name__"] = mod.__name__
    exec(compile(src.replace(old, new), ow.__file__, "exec"), mod.__dict__)
    caught = False
    for a in MAPS[:2]:
        try:
            M = mod.covariance(a, 0.6) - 0.36 * np.eye(2)
            J = np.array([[a[0], a[1]], [a[3], a[4]]])
            s = np.random.default_rng(5).normal(size=(40, 2))
            lhs = np.einsum("ni,ij,nj->n", s, np.linalg.inv(M), s)
            rhs = (np.linalg.solve(J, s.T).T ** 2).sum(1) / 0.36
            assert np.abs(lhs - rhs).max() < 1e-10 * rhs.max()
            img = np.random.default_rng(7).random((9, 11))
            out = mod.warp(img, 7, 8, a, 0.6, 3.0, "clamp")
            assert np.abs(out - ewa_independent(img, 7, 8, a, 0.6, 3.0)).max() < 1e-9
        except (AssertionError, np.linalg.LinAlgError):
            caught = True
            break
    assert caught, "no pin caught warp mutant %s" % name
