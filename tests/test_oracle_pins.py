"""The FP64 oracle against closed forms, published kernel values, numpy.pad,
torch's float64 interpolate, an exact-rational brute force and invariants."""
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=[p.__name__ for p in pins.ALL_PINS])
def test_pin(o, pin):
    pin(o)


@pytest.mark.parametrize("n_in,n_out", [(97, 41), (41, 97), (4096, 1229), (13, 13)])
@pytest.mark.parametrize("kernel,param", [("lanczos", 3.0), ("cubic", -0.5), ("gaussian", 0.7)])
def test_mirror_outputs_take_reversed_weights(o, n_in, n_out, kernel, param):
    """Half-pixel centres make the grid symmetric: output n_out-1-i sits where
    output i sits seen from the other end, so with a symmetric kernel and the
    clamp map its raw taps are those of output i mirrored (j -> n_in-1-j) and
    its weights the same values in reverse order."""
    for i in list(range(6)) + [n_out // 2]:
        jf, idx, w = o.axis_weights_at(n_in, n_out, kernel, "clamp", i, param=param)
        jm, idxm, wm = o.axis_weights_at(n_in, n_out, kernel, "clamp", n_out - 1 - i, param=param)
        assert jm == n_in - jf - len(w)
        assert (idxm[::-1] == n_in - 1 - idx).all()
        assert abs(wm[::-1] - w).max() < 1e-15


def test_single_output_weights_match_the_rows(o):
    rows = o.axis_weights(50, 17, "lanczos", "mirror", param=3.0)
    for i, (jf, idx, w) in enumerate(rows):
        jf2, idx2, w2 = o.axis_weights_at(50, 17, "lanczos", "mirror", i, param=3.0)
        assert jf2 == jf and (idx2 == idx).all() and (w2 == w).all()
