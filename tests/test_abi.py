"""Host-side checks of the C ABI: the library loads, exports exactly what
include/nh.h declares, and validates parameters without touching a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "nh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nh_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def nh():
    from paper_2503_06610_gb300 import nh as m
    m.load_library()
    return m


def test_library_exports_every_declared_symbol(nh):
    lib = nh.load_library()
    decl = _declared()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(nh.SIGNATURES) == decl


def test_params_struct_layout_matches_header(nh):
    import ctypes
    # 16 int32 then 18 doubles, no padding; the reading flags follow frank3
    assert ctypes.sizeof(nh.nh_params) == 16 * 4 + 18 * 8
    assert nh.nh_params.tau.offset == 64
    names = [f[0] for f in nh.nh_params._fields_]
    assert names[11:16] == ["frank3", "renorm_predictor", "lap_wide", "n_from_rate", "ghost_sigma"]


def _base(**kw):
    d = dict(nx=8, ny=8, nz=8, precision="fp32", tau=1.0, gamma1=1.0, dt_fd=1)
    d.update(kw)
    return d


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(tau=0.5), dict(tau=0.2), dict(gamma1=0.0), dict(dt_fd=0),
    dict(precision="fp64", storage="f32"), dict(precision="fp32", storage="f64"),
    dict(storage="f16s", shifted=False), dict(storage="bf16s", shifted=False),
    dict(K=float("nan")), dict(nx=2000, ny=2000, nz=100),
    dict(K=0.04, dt_fd=8, check_stability=True),
    dict(K11=0.0, K22=1.0, K33=1.0), dict(K11=1.0, K22=float("inf"), K33=1.0),
    dict(nx=113025456, ny=1, nz=1),
    dict(renorm_predictor=2), dict(lap_wide=-1), dict(n_from_rate=3), dict(ghost_sigma=2),
])
def test_invalid_params_rejected(nh, bad):
    p = nh.make_params(_base(**bad))
    with pytest.raises(nh.NHError) as e:
        nh.nh_workspace_bytes(p)
    assert e.value.code == nh.NH_EINVAL


def test_largest_domain_accepted(nh):
    """19 N must fit a signed 32-bit index: N = 113 025 455 is the largest channel."""
    assert nh.nh_workspace_bytes(nh.make_params(_base(nx=113025455, ny=1, nz=1))) > 19 * 4 * 113025455


def test_workspace_size_formula(nh):
    N = 8 * 8 * 8
    b32 = nh.nh_workspace_bytes(nh.make_params(_base()))
    b16 = nh.nh_workspace_bytes(nh.make_params(_base(storage="f16s")))
    b64 = nh.nh_workspace_bytes(nh.make_params(_base(precision="fp64")))
    assert b32 - b16 >= 2 * 19 * N * 2 - 2 * 256
    assert b64 > b32
    assert nh.nh_workspace_bytes(nh.make_params(_base(K=0.04, dt_fd=4, check_stability=True))) > 0


def test_error_strings(nh):
    lib = nh.load_library()
    assert lib.nh_error_string(nh.NH_EINVAL) == b"invalid argument"
    assert lib.nh_error_string(nh.NH_EUNSTABLE)
    assert lib.nh_last_error(None) is not None
