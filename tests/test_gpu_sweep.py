"""The precision / dt_FD behaviour the paper reports (Secs. III.A-III.B), in kind,
on a small skyrmion channel through the CUDA path:

* in FP64 the error against the dt_FD = 1 run grows monotonically with dt_FD
  (Sec. III.A: "increases monotonically");
* in FP32 at low velocity the shifted populations are more accurate than the
  plain ones (Sec. II.C, Sec. III.A).
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sweep_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import sweep
    return sweep


def test_fp64_error_grows_with_dt_fd(sweep_mod):
    res = sweep_mod.sweep(steps=480, gx=1e-5, dts=(1, 2, 4, 8), settings=[("fp64", "f64", True)],
                          nx=32, ny=32, nz=16, radius=6.0)
    errs = [r["eps_u"] for r in res["rows"]]
    nerr = [r["rel_l2_n"] for r in res["rows"]]
    assert errs[0] == 0.0
    assert all(b > a for a, b in zip(errs[1:], errs[2:]))
    assert all(b > a for a, b in zip(nerr[1:], nerr[2:]))
    assert all(r["nonfinite"] == 0 for r in res["rows"])


def test_shift_reduces_fp32_error_at_low_velocity(sweep_mod):
    settings = [("fp64", "f64", True), ("fp32", "f32", False), ("fp32", "f32", True)]
    res = sweep_mod.sweep(steps=400, gx=1e-7, dts=(4,), settings=settings, nx=32, ny=32, nz=16, radius=6.0)
    rows = {(r["precision"], r["shifted"]): r for r in res["rows"]}
    ref = rows[("fp64", True)]
    plain = rows[("fp32", False)]
    shifted = rows[("fp32", True)]
    # errors are measured against the FP64 dt_FD = 1 run; subtract the FP64 dt_FD = 4 part
    assert shifted["eps_u"] < plain["eps_u"]
    assert abs(shifted["eps_u"] - ref["eps_u"]) < abs(plain["eps_u"] - ref["eps_u"])
