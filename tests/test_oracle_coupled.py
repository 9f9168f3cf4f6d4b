"""Pins of the oracle's coupled hybrid loop (Secs. II.A-II.D of arXiv:2503.06610).

The size of the backflow around a distorted director has no closed form, but
two balance laws of the continuum equations hold for the coupled loop and
involve every coupling term at once:

* energy: with no body force, resting no-slip plates and held (or free)
  anchoring, the Ericksen-Leslie equations dissipate: the kinetic energy of
  the flow plus the Frank energy of the director never increases when the
  Leslie coefficients satisfy Leslie's inequalities.  The flow -> director
  terms (advection, co-rotation, flow alignment) and the director -> flow
  terms (elastic and viscous stress through the force divergence) only trade
  energy, so a wrong sign or a transposed index in either direction makes the
  total rise.  The discrete loop keeps the law step by step at dt_FD = 1, and
  from one FD interval to the next at larger dt_FD within the Heun limit
  (within an interval the held force does work the director does not answer);
* momentum: in a fully periodic box the force is the discrete divergence of
  the stress and sums to zero over the lattice, so the total momentum of the
  populations changes by exactly the body force times the mass per step.

Planted mistakes (composed from the oracle's routines on the CPU) show that
the energy law fails for each of: force of the wrong sign, the stress's two
indices exchanged, the flow's sign flipped in the director equation, and the
Leslie coefficients alpha2 and alpha3 exchanged in the stress.
"""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

LES = I.LESLIE_DISSIPATIVE
SHAPE = (12, 12, 8)


def _params(O, **kw):
    nx, ny, nz = SHAPE
    d = dict(nx=nx, ny=ny, nz=nz, walls_z=False, anchoring="homeotropic", shifted=True, tau=1.0,
             g=(0.0, 0.0, 0.0), K=0.04, q0=0.0, W0=0.0, dt_fd=1, **LES)
    d.update(kw)
    return O.OracleParams.from_dict(d)


def _total_energy(O, p, rho, u, n):
    return 0.5 * float(np.sum(rho * np.sum(u * u, axis=0))) + O.frank_energy(p, n)


def test_leslie_inequalities_hold_for_the_dissipative_set():
    """alpha4 of the LB fluid at tau = 1 is 2 rho nu = 2 (tau - 1/2)/3 (alpha4' = 0)."""
    a1, a2, a3, a5, a6 = (LES[k] for k in ("alpha1", "alpha2", "alpha3", "alpha5", "alpha6"))
    a4 = 2 * (1.0 - 0.5) / 3 + LES["alpha4p"]
    g1, g2 = a3 - a2, a3 + a2
    assert abs(g1 - LES["gamma1"]) < 1e-15 and abs(g2 - LES["gamma2"]) < 1e-15
    assert abs((a6 - a5) - g2) < 1e-15  # Parodi
    assert a4 > 0 and g1 > 0
    assert 2 * a1 + 3 * a4 + 2 * a5 + 2 * a6 > 0
    assert 2 * a4 + a5 + a6 > 0
    assert 4 * g1 * (2 * a4 + a5 + a6) > (a2 + a3 + a6 - a5) ** 2
    # the flow-aligning set of the channel workloads does not satisfy the last one
    L = I.LESLIE_ALIGN_09
    assert 4 * L["gamma1"] * (2 * a4 + L["alpha5"] + L["alpha6"]) < (L["alpha2"] + L["alpha3"] + L["alpha6"]
                                                                    - L["alpha5"]) ** 2


@pytest.mark.parametrize("walls,anchoring,q0,W0,shifted", [
    (False, "homeotropic", 0.0, 0.0, True),
    (True, "homeotropic", 0.0, 0.0, True),
    (True, "none", 0.0, 0.0, True),
    (True, "none", 2 * math.pi / 8, 0.01, True),
    (False, "homeotropic", 2 * math.pi / 8, 0.0, False),
])
def test_coupled_total_energy_dissipates_each_step(oracle_mod, walls, anchoring, q0, W0, shifted):
    O = oracle_mod
    p = _params(O, walls_z=walls, anchoring=anchoring, q0=q0, W0=W0, shifted=shifted)
    sim = O.OracleSim(p, I.distorted_director(*SHAPE))
    E = [_total_energy(O, p, sim.rho, sim.u, sim.n)]
    umax = 0.0
    for _ in range(200):
        sim.step(1)
        E.append(_total_energy(O, p, sim.rho, sim.u, sim.n))
        umax = max(umax, float(np.max(np.abs(sim.u))))
    dE = np.diff(E)
    assert np.all(dE < 0.0), (dE.max(), int(np.argmax(dE)))
    assert E[-1] < 0.9 * E[0]
    assert umax > 1e-3  # the backflow is not negligible: the coupling terms carry energy


@pytest.mark.parametrize("dt_fd", [2, 4])
@pytest.mark.parametrize("walls", [False, True])
def test_coupled_total_energy_dissipates_each_fd_interval(oracle_mod, dt_fd, walls):
    O = oracle_mod
    p = _params(O, walls_z=walls, dt_fd=dt_fd)
    assert dt_fd * 6 * p.K / p.gamma1 < 1  # within the Heun limit of the compact Laplacian
    sim = O.OracleSim(p, I.distorted_director(*SHAPE))
    E = [_total_energy(O, p, sim.rho, sim.u, sim.n)]
    for _ in range(240 // dt_fd):
        sim.step(dt_fd)
        E.append(_total_energy(O, p, sim.rho, sim.u, sim.n))
    dE = np.diff(E)
    assert np.all(dE < 0.0), (dE.max(), int(np.argmax(dE)))


def _composed_run(O, p, steps, stress_fn, fd_fn):
    """The fused-order loop of OracleSim at dt_FD = 1 written out from the oracle's routines."""
    sim = O.OracleSim(p, I.distorted_director(*SHAPE))
    sim.F = O.force(p, stress_fn(sim.n, sim.u))
    E = []
    for _ in range(steps):
        sim.f, sim.rho, sim.u = O.lb_step(p, sim.f, sim.F)
        sim.n = fd_fn(sim.n, sim.u)
        sim.F = O.force(p, stress_fn(sim.n, sim.u))
        E.append(_total_energy(O, p, sim.rho, sim.u, sim.n))
    return sim, np.array(E)


def test_energy_law_fails_for_planted_coupling_mistakes(oracle_mod):
    O = oracle_mod
    p = _params(O)
    steps = 120
    ref = O.OracleSim(p, I.distorted_director(*SHAPE)).step(steps)
    sim, E = _composed_run(O, p, steps, lambda n, u: O.stress(p, n, u), lambda n, u: O.fd_step(p, n, u))
    assert np.array_equal(sim.n, ref.n) and np.array_equal(sim.u, ref.u)
    assert np.all(np.diff(E) < 0.0)

    def transposed(s):
        return s.reshape(3, 3, -1).transpose(1, 0, 2).reshape(9, -1)

    p23 = O.OracleParams.from_dict(dict(p.__dict__, alpha2=LES["alpha3"], alpha3=LES["alpha2"]))
    planted = {
        "force sign": (lambda n, u: -O.stress(p, n, u), lambda n, u: O.fd_step(p, n, u)),
        "stress indices exchanged": (lambda n, u: transposed(O.stress(p, n, u)), lambda n, u: O.fd_step(p, n, u)),
        "flow sign in the director equation": (lambda n, u: O.stress(p, n, u), lambda n, u: O.fd_step(p, n, -u)),
        "alpha2 and alpha3 exchanged in the stress": (lambda n, u: O.stress(p23, n, u),
                                                      lambda n, u: O.fd_step(p, n, u)),
    }
    for name, (sf, ff) in planted.items():
        _, Ep = _composed_run(O, p, steps, sf, ff)
        assert np.max(np.diff(Ep)) > 1e-3 * E[0], name


@pytest.mark.parametrize("g", [(0.0, 0.0, 0.0), (2e-6, -1e-6, 5e-7)])
def test_coupled_momentum_balance_periodic(oracle_mod, g):
    """Total population momentum after s steps = s * M * g, M the (conserved) mass."""
    O = oracle_mod
    p = _params(O, g=g, q0=2 * math.pi / 8)
    e, _, _ = O.lattice()
    sim = O.OracleSim(p, I.distorted_director(*SHAPE))
    M = float(np.sum(sim.rho))
    scale = 0.0
    for s in range(1, 161):
        sim.step(1)
        mom = e.T.astype(np.float64) @ sim.f.reshape(19, -1).sum(axis=1)
        expect = s * M * np.asarray(g)
        scale = max(scale, float(np.sum(np.abs(sim.rho * sim.u))))
        assert np.max(np.abs(mom - expect)) <= 1e-12 * max(scale, 1e-3), (s, mom, expect)
    assert scale > 1e-2  # local momenta far above the allowance
