"""Planted mistakes: each test compiles a copy of the oracle with one
plausible bug (a sign, an index, a dropped term, a transposed operand) on the
CPU and checks that at least one pin in ``pins.py`` rejects it."""
import os

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")

# (name, text to replace, replacement) -- each replacement must apply once.
MUTANTS = [
    ("keys_sign", "- (a + 3.0) * t * t + 1.0", "+ (a + 3.0) * t * t - 1.0"),
    ("keys_outer_term", "+ 8.0 * a * t - 4.0 * a", "+ 8.0 * a * t + 4.0 * a"),
    ("mirror_off_by_one", "return m < n ? m : p - 1 - m;", "return m < n ? m : p - m;"),
    ("reflect101_as_mirror", "return m < n ? m : p - m;\n", "return m < n ? m : p - 1 - m;\n"),
    ("clamp_edge", "return j < 0 ? 0 : (j >= n ? n - 1 : j);", "return j < 0 ? 0 : (j >= n ? n - 2 : j);"),
    ("no_antialias_widening", "if (antialias && n_in > n_out) return 2 * n_in;",
     "if (antialias && n_in > n_out) return 2 * n_out;"),
    ("no_normalisation", "for (int64_t k = 0; k < n; ++k) w[k] = w[k] / sum;", "(void)sum;"),
    ("centre_half_pixel_dropped",
     "        int64_t num = (2 * j + 1) * n_out - (2 * i + 1) * n_in;\n        double x",
     "        int64_t num = (2 * j) * n_out - (2 * i) * n_in;\n        double x"),
    ("lanczos_window_dropped", "return ora_sinc(x) * ora_sinc(x / R);", "return ora_sinc(x);"),
    ("bspline_cubic_term", "2.0 / 3.0 - t * t + t * t * t / 2.0", "2.0 / 3.0 - t * t + t * t * t / 3.0"),
    ("support_not_strict", "if (num < R * D) {", "if (num <= R * D) {"),
    ("row_stride_transposed", "const double *irow = J->in + idx_h[ty] * J->in_w * J->ch;",
     "const double *irow = J->in + idx_h[ty] * J->in_h * J->ch;"),
    ("weights_axes_swapped", "acc += wt_h[ty] * wx[tx] * irow[ix[tx] * J->ch + c];",
     "acc += wt_h[tx < n ? tx : ty] * wx[tx] * irow[ix[tx] * J->ch + c];"),
    ("truncate_keeps_weight", "w[k] = (m < 0) ? 0.0 : ora_kernel_value(kernel, param, x);",
     "w[k] = ora_kernel_value(kernel, param, x);"),
    ("sinc_sign", "return (fmod(k, 2.0) != 0.0) ? -s : s;", "return s;"),
    ("mitchell_c_relation", "double B = param, C = (1.0 - B) / 2.0;", "double B = param, C = (1.0 - B) / 3.0;"),
    ("mitchell_outer_term", "(-12.0 * B - 48.0 * C) * t +", "(-12.0 * B - 46.0 * C) * t +"),
    ("gaussian_width", "return exp(-(x * x) / (2.0 * param * param));", "return exp(-(x * x) / (param * param));"),
    ("gaussian_no_truncation", "        if (t >= R) return 0.0;\n        return exp(",
     "        (void)R;\n        return exp("),
]

# fast pins first; the exhaustive tap scan last
ORDER = [pins.pin_kernel_values, pins.pin_keys_x2, pins.pin_bilinear_aa_half, pins.pin_identity,
         pins.pin_constant, pins.pin_polynomials, pins.pin_polynomial_image, pins.pin_boundary_pad,
         pins.pin_invariants, pins.pin_mitchell_gaussian, pins.pin_brute, pins.pin_torch,
         pins.pin_taps_fractions]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not unique: %s" % name
    mutant = tmp_path / ("rs_oracle_%s.c" % name)
    mutant.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(mutant), out=str(tmp_path / ("lib_%s.so" % name)))
    o = oracle.Oracle(lib)
    failed = None
    for pin in ORDER:
        try:
            pin(o)
        except (AssertionError, ValueError) as e:  # ValueError: the oracle refused
            failed = (pin.__name__, e)
            break
    assert failed is not None, "no pin caught mutant %s" % name
