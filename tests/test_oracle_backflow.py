"""The size of the coupled backflow in the oracle's hybrid loop, against the
linear theory of the Ericksen-Leslie equations (Secs. II.A-II.C of
arXiv:2503.06610).

A small director wave in a fully periodic box couples to a shear flow.  With
the director n0 + delta n, delta n = N(t) sin(kz) e_p, and the flow
u = V(t) cos(kz) e_x, the linearised equations close on (N, V):

* bend geometry, n0 = z_hat, e_p = x_hat (coefficients alpha2, alpha5):
    dN/dt = -(K/g1) L N + (a2/g1) s V
    dV/dt = -(nu k^2 + eta_fd s^2) V - (a2 K/g1) s L N,
    eta_fd = (a4' + a5)/2 - a2 g2/(2 g1);
* splay geometry, n0 = x_hat, e_p = z_hat: the same with alpha2 -> alpha3 and
  alpha5 -> alpha6.

The director rows come from the director equation (the flow alignment
-lambda D.n and the co-rotation W.n), the flow rows from the LB's Newtonian
viscosity nu = (tau - 1/2)/3 and the divergence of the Leslie stress
sigma_xz = alpha_{2|3} N + (alpha4' + alpha_{5|6}) du_x/dz / 2, with the
kinematic transport N taken from the director equation.  The lattice enters
only through the symbols of the central first derivative (s = sin k) and of
the compact Laplacian (L = 4 sin^2(k/2)); the LB's shear viscosity is taken
at its continuum value.  The oracle follows the solution of this 2 x 2 system
(a decaying oscillation for the dissipative coefficients) to 1e-3 of the
initial amplitude, and its deviation falls by k^2 when the wave is made twice
as long; a stress off by 10 % misses it by several percent.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from paper_2503_06610_gb300 import inputs as I

LES = I.LESLIE_DISSIPATIVE
K, TAU, AMP, NXY = 0.04, 1.0, 1e-3, 2


def _params(O, nz):
    return O.OracleParams.from_dict(dict(nx=NXY, ny=NXY, nz=nz, walls_z=False, anchoring="homeotropic",
                                         shifted=True, tau=TAU, g=(0.0, 0.0, 0.0), K=K, q0=0.0, W0=0.0, dt_fd=1,
                                         **LES))


def _start(nz, geometry):
    N = NXY * NXY * nz
    z = np.arange(N) // (NXY * NXY)
    wave = AMP * np.sin(2 * math.pi * z / nz)
    one, zero = np.ones(N), np.zeros(N)
    n0 = np.stack([wave, zero, one]) if geometry == "bend" else np.stack([one, zero, wave])
    return n0 / np.linalg.norm(n0, axis=0), z


def _theory(nz, geometry, times, N0):
    k = 2 * math.pi / nz
    s, L = math.sin(k), 4 * math.sin(k / 2) ** 2
    g1, g2, a4p = LES["gamma1"], LES["gamma2"], LES["alpha4p"]
    a, a56 = (LES["alpha2"], LES["alpha5"]) if geometry == "bend" else (LES["alpha3"], LES["alpha6"])
    nu = (TAU - 0.5) / 3
    eta_fd = (a4p + a56) / 2 - a * g2 / (2 * g1)
    M = np.array([[-K * L / g1, a * s / g1],
                  [-a * K * s * L / g1, -(nu * k * k + eta_fd * s * s)]])
    sol = np.array([expm(M * t) @ np.array([N0, 0.0]) for t in times])
    return sol[:, 0], sol[:, 1], np.linalg.eigvals(M)


def _amplitudes(sim, z, nz, geometry):
    k = 2 * math.pi / nz
    S, C = np.sin(k * z), np.cos(k * z)
    comp = 0 if geometry == "bend" else 2
    return np.sum(sim.n[comp] * S) / np.sum(S * S), np.sum(sim.u[0] * C) / np.sum(C * C)


def _run(O, nz, geometry, steps, every, stress_scale=None):
    p = _params(O, nz)
    n0, z = _start(nz, geometry)
    sim = O.OracleSim(p, n0)
    times, Ns, Vs = [0], [], []
    a0 = _amplitudes(sim, z, nz, geometry)
    Ns.append(a0[0])
    Vs.append(a0[1])
    if stress_scale is not None:  # planted: the force of a stress off by a factor, same loop as OracleSim
        sim.F = O.force(p, stress_scale * O.stress(p, sim.n, sim.u))
    for q in range(steps // every):
        for _ in range(every):
            if stress_scale is None:
                sim.step(1)
            else:
                sim.f, sim.rho, sim.u = O.lb_step(p, sim.f, sim.F)
                sim.n = O.fd_step(p, sim.n, sim.u)
                sim.F = O.force(p, stress_scale * O.stress(p, sim.n, sim.u))
        times.append((q + 1) * every)
        a = _amplitudes(sim, z, nz, geometry)
        Ns.append(a[0])
        Vs.append(a[1])
    return np.array(times), np.array(Ns), np.array(Vs)


@pytest.mark.parametrize("geometry", ["bend", "splay"])
def test_coupled_mode_follows_linear_theory(oracle_mod, geometry):
    O = oracle_mod
    errs = []
    for nz, steps in ((64, 4000), (128, 12000)):
        t, Ns, Vs = _run(O, nz, geometry, steps, 200)
        Np, Vp, ev = _theory(nz, geometry, t, Ns[0])
        assert np.all(ev.real < 0)  # Leslie's inequalities hold: the mode decays
        eN = np.max(np.abs(Ns - Np)) / abs(Ns[0])
        eV = np.max(np.abs(Vs - Vp)) / np.max(np.abs(Vp))
        assert eN < 1e-3 and eV < 2e-3, (nz, eN, eV)
        # the backflow matters: the coupled decay rate is far from the director's own K L / g1
        bare = K * 4 * math.sin(math.pi / nz) ** 2 / LES["gamma1"]
        assert abs(-ev.real.max() - bare) > 0.3 * bare
        errs.append(eN)
    assert errs[1] < 0.4 * errs[0]  # second-order convergence in the wavelength


def test_bend_mode_oscillates_and_decays_as_predicted(oracle_mod):
    """Dissipative bend mode at nz = 64: a damped oscillation (complex eigenvalues),
    and the oracle's amplitude crosses zero where the theory says."""
    O = oracle_mod
    t, Ns, _ = _run(O, 64, "bend", 4000, 100)
    Np, _, ev = _theory(64, "bend", t, Ns[0])
    assert np.all(np.abs(ev.imag) > 1e-4)
    sign_change = lambda a: int(np.argmax(np.sign(a) != np.sign(a[0])))
    assert sign_change(Ns) == sign_change(Np) > 0


def test_stress_off_by_ten_percent_misses_the_mode(oracle_mod):
    O = oracle_mod
    t, Ns, _ = _run(O, 64, "bend", 4000, 200, stress_scale=1.1)
    Np, _, _ = _theory(64, "bend", t, Ns[0])
    assert np.max(np.abs(Ns - Np)) / abs(Ns[0]) > 2e-2
