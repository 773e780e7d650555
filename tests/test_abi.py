"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol include/rs.h declares, and rejects malformed descriptors before it
touches a GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rs():
    from conftest import load_build_module

    load_build_module().build()
    import paper_1110_5450_b300 as rs

    return rs


def header_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:RS_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(rs_[a-z0-9_]+)\s*\(", text,
                            flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = header_functions()
    for n in ("rs_plan_create", "rs_resample", "rs_destroy", "rs_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(rs):
    lib = ctypes.CDLL(rs.LIB_PATH)
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(header_functions()) <= set(rs.EXPORTS) | set(header_functions())


def test_binding_covers_header(rs):
    assert set(header_functions()) == set(rs.EXPORTS)


def test_status_strings(rs):
    for code in range(9):
        assert rs.rs_status_string(code)
    assert rs.rs_version() >= 1


def _desc(rs, **kw):
    base = dict(in_h=16, in_w=16, channels=1, out_h=8, out_w=8, kernel="cubic", boundary="clamp",
                dtype=rs.RS_F32)
    base.update(kw)
    return rs.make_desc(**base)


@pytest.mark.parametrize("bad", [
    dict(in_h=0), dict(in_w=-3), dict(channels=0), dict(channels=65), dict(out_h=-1),
    dict(in_h=1 << 23), dict(out_h=0, scale_h=0.0), dict(out_w=0, scale_w=float("nan")),
    dict(kernel="lanczos", param=2.5), dict(kernel="lanczos", param=0.0), dict(flags=0x200),
    dict(kernel="mitchell", param=1.5), dict(kernel="gaussian", param=0.0),
    dict(in_row_stride=5),
])
def test_invalid_descriptors_rejected_without_gpu(rs, bad):
    d = _desc(rs, **bad)
    with pytest.raises(rs.RSError) as ei:
        rs.rs_plan_create(d, 0)
    assert ei.value.status == rs.RS_ERR_INVALID_ARG, str(ei.value)


@pytest.mark.parametrize("bad", [dict(kernel="lanczos"), dict(kernel="bspline3", boundary="truncate"),
                                 dict(kernel="bspline3", dtype=3)])
def test_prefilter_misuse_rejected_without_gpu(rs, bad):
    """RS_PREFILTER takes the cubic B-spline, FP32/FP64 and a symmetric or clamped boundary."""
    d = _desc(rs, flags=rs.RS_PREFILTER, **bad)
    with pytest.raises(rs.RSError) as ei:
        rs.rs_plan_create(d, 0)
    assert ei.value.status == rs.RS_ERR_UNSUPPORTED, str(ei.value)


def test_unknown_enum_and_dtype_mismatch(rs):
    d = _desc(rs)
    d.kernel = 9
    with pytest.raises(rs.RSError) as ei:
        rs.rs_plan_create(d, 0)
    assert ei.value.status == rs.RS_ERR_INVALID_ARG
    d = _desc(rs)
    d.out_dtype = rs.RS_F16
    with pytest.raises(rs.RSError) as ei:
        rs.rs_plan_create(d, 0)
    assert ei.value.status == rs.RS_ERR_UNSUPPORTED


def test_too_many_taps_is_unsupported(rs):
    d = _desc(rs, in_h=4096, in_w=16, out_h=2, out_w=8, kernel="lanczos", param=3)
    with pytest.raises(rs.RSError) as ei:
        rs.rs_plan_create(d, 0)
    assert ei.value.status == rs.RS_ERR_UNSUPPORTED


def test_null_arguments(rs):
    lib = ctypes.CDLL(rs.LIB_PATH)
    lib.rs_plan_create.restype = ctypes.c_int
    assert lib.rs_plan_create(None, None, None) == rs.RS_ERR_INVALID_ARG
    assert lib.rs_resample(None, None, None, None) == rs.RS_ERR_INVALID_ARG
    assert lib.rs_destroy(None) == rs.RS_OK


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1110_5450_b300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f
                assert "liboracle" not in text and "rs_oracle" not in text, f
