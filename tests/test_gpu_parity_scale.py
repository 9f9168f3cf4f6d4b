"""Parity at the size of the single-tube workload, element by element, and the
paper's own regime at its own dt_FD.

* 96x96x32 skyrmion tube in Poiseuille flow between homeotropic plates
  (q0 = 2 pi/32, R = 12, g_x = 1e-5): the FP64 GPU path against the oracle
  after 200 LB steps at dt_FD = 1 and 4, as rel. L2 and as the largest
  per-site difference of u and n, with the two plate layers checked by name.
* The Table I regime (Sec. III.A: 64x64x16, g = 2e-9, no plate anchoring,
  equal viscosity shares in the LB and the FD force) in the loop order of
  Sec. II.D at dt_FD = 1, the paper's reference setting: stays finite with
  the velocity of plain Poiseuille flow (~1e-7) (the fused order diverges).
"""
import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import nh as m
    m.load_library()
    return m


def _layers(a, nz):
    return np.asarray(a).reshape(3, nz, -1)


@pytest.mark.parametrize("dt_fd", [1, 4])
def test_skyrmion_channel_fp64_per_element(nh, oracle_mod, dt_fd):
    O = oracle_mod
    params, n0 = I.skyrmion_channel(gx=1e-5, dt_fd=dt_fd)
    nz = params["nz"]
    ref = O.OracleSim(O.OracleParams.from_dict(params), n0).step(200)
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fields(n0)
    ch.step(200)
    n, u, rho = ch.get_fields()
    f = ch.get_populations()
    umax = float(np.max(np.abs(ref.u)))
    assert umax > 1e-4  # the flow and the backflow are developed
    assert O.rel_l2(u, ref.u) <= 1e-10
    assert O.rel_l2(n, ref.n) <= 1e-10
    assert np.max(np.abs(u - ref.u)) <= 1e-10 * umax
    assert np.max(np.abs(n - ref.n)) <= 1e-12
    assert np.max(np.abs(rho - ref.rho)) <= 1e-14
    assert np.max(np.abs(f - ref.f)) <= 1e-14
    du, dn = _layers(u - ref.u, nz), _layers(n - ref.n, nz)
    for z, name in ((0, "lowest plate layer"), (nz - 1, "highest plate layer")):
        assert np.max(np.abs(du[:, z])) <= 1e-10 * umax, name
        assert np.max(np.abs(dn[:, z])) <= 1e-12, name
    d = ch.diagnostics()
    assert abs(d["energy"] - ref.energy()) <= 1e-11 * abs(ref.energy())
    ch.close()


def test_table1_regime_paper_order_dt1_stable(nh):
    params, n0 = I.table1_regime(dt_fd=1, split=0.5)  # equal viscosity shares in LB and FD, Sec. II.B
    assert params["paper_order"] and abs(params["alpha4p"] - 0.5 * 0.9318) < 1e-12
    ch = nh.Channel(dict(params, precision="fp32", storage="f32"))
    ch.set_fields(n0)
    peak = 0.0
    for _ in range(10):
        ch.step(10000)
        _, u, _ = ch.get_fields()
        assert np.all(np.isfinite(u))
        peak = max(peak, float(np.max(np.abs(u))))
    assert 1e-8 < peak < 1e-6
    d = ch.diagnostics()
    assert d["nonfinite"] == 0
    ch.close()
