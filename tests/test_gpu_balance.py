"""Balance laws of the coupled CUDA loop (through the C ABI) at sizes beyond the oracle's reach.

The same laws pin the oracle's coupled loop (tests/test_oracle_coupled.py):
with Leslie coefficients that satisfy Leslie's inequalities and no body
force, the kinetic plus Frank energy of the Ericksen-Leslie equations never
increases (Secs. II.A-II.B), step by step at dt_FD = 1 and from one FD
interval to the next at larger dt_FD; in a fully periodic box the population
momentum after s steps is s M g, because the force is an exact discrete
divergence (Sec. II.C, Guo forcing).  Both FD kernel variants (fused 2.5D and
per-site) and both arithmetic precisions are held to them.
"""
import math

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


def _channel(nh, shape, precision, storage, fused, **kw):
    nx, ny, nz = shape
    params = dict(nx=nx, ny=ny, nz=nz, walls_z=False, anchoring="homeotropic", shifted=True, tau=1.0,
                  g=(0.0, 0.0, 0.0), K=0.04, q0=0.0, W0=0.0, dt_fd=1, precision=precision, storage=storage,
                  **I.LESLIE_DISSIPATIVE)
    params.update(kw)
    ch = nh.Channel(params)
    ch.set_fd_variant(fused)
    ch.set_fields(I.distorted_director(nx, ny, nz))
    return ch


def _total_energy(ch):
    _, u, rho = ch.get_fields()
    return 0.5 * float(np.sum(rho * np.sum(u * u, axis=0))) + ch.diagnostics()["energy"]


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("precision,storage", [("fp64", "f64"), ("fp32", "f32")])
@pytest.mark.parametrize("shape,kw", [
    ((64, 64, 32), dict()),
    ((48, 40, 24), dict(walls_z=True, anchoring="homeotropic")),
    ((48, 40, 24), dict(walls_z=True, anchoring="none", q0=2 * math.pi / 24, W0=0.002)),
])
def test_coupled_energy_dissipates_each_step(nh, shape, kw, precision, storage, fused):
    ch = _channel(nh, shape, precision, storage, fused, **kw)
    try:
        E = [_total_energy(ch)]
        umax = 0.0
        for _ in range(150):
            ch.step(1)
            E.append(_total_energy(ch))
            umax = max(umax, ch.diagnostics()["max_u"])
        dE = np.diff(E)
        assert np.all(dE < 0.0), (dE.max(), int(np.argmax(dE)))
        assert E[-1] < 0.97 * E[0]
        assert umax > 1e-5
    finally:
        ch.close()


@pytest.mark.parametrize("fused", [1, 0])
def test_coupled_energy_dissipates_each_fd_interval(nh, fused):
    dt_fd = 4
    ch = _channel(nh, (64, 48, 32), "fp32", "f32", fused, walls_z=True, dt_fd=dt_fd)
    try:
        E = [_total_energy(ch)]
        for _ in range(40):
            ch.step(dt_fd)
            E.append(_total_energy(ch))
        dE = np.diff(E)
        assert np.all(dE < 0.0), (dE.max(), int(np.argmax(dE)))
    finally:
        ch.close()


@pytest.mark.parametrize("precision,storage,tol", [("fp64", "f64", 1e-11), ("fp32", "f32", 1e-5)])
def test_coupled_momentum_balance_periodic(nh, oracle_mod, precision, storage, tol):
    g = np.array([2e-6, -1e-6, 5e-7])
    shape = (64, 64, 32)
    ch = _channel(nh, shape, precision, storage, 1, g=tuple(g), q0=2 * math.pi / 32)
    try:
        e = oracle_mod.lattice()[0].astype(np.float64)  # the population order both sides share
        M = float(np.sum(ch.get_fields()[2]))
        s = 0
        scale = 0.0
        for chunk in (1, 7, 24, 64):
            ch.step(chunk)
            s += chunk
            f = ch.get_populations()
            mom = e.T @ f.sum(axis=1)
            _, u, rho = ch.get_fields()
            scale = max(scale, float(np.sum(np.abs(rho * u))))
            assert np.max(np.abs(mom - s * M * g)) <= tol * scale, (s, mom, s * M * g)
        assert scale > 1.0
    finally:
        ch.close()
