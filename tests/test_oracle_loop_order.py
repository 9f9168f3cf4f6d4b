"""The loop order of Sec. II.D decides whether the paper's own regime is stable.

In the Table I regime (MBBA viscosities, the same isotropic viscosity in the
LB and in the FD force as Sec. II.B chooses) the hybrid loop in its printed
order -- macroscopic fields, FD update and force, then the collision of the
same step -- is stable at dt_FD = 1.  The fused order, whose collision keeps
the force of the previous interval, lets the force lag the velocity it is
computed from by one LB step; at odd dt_FD the lag feeds a lattice mode that
flips sign every step (k_x = k_y = pi/2 and about the same k_z, where the central
differences of the viscous stress are largest) and the run diverges.  Both
runs are oracle runs on a small channel with plates; nothing here touches the
GPU path.
"""
import numpy as np

from paper_2503_06610_gb300 import inputs as I


def _sim(O, paper_order, dt_fd=1, g=None):
    p, _ = I.table1_regime(nx=8, ny=8, nz=16, dt_fd=dt_fd, split=0.5, paper_order=paper_order)
    if g is not None:
        p = dict(p, g=g)
    n0 = I.tilted_director(8, 8, 16, amplitude=0.05, seed=1)
    return O.OracleSim(O.OracleParams.from_dict(p), n0)


def test_paper_order_is_stable_at_dt1(oracle_mod):
    sim = _sim(oracle_mod, True)
    peak = 0.0
    for _ in range(6):
        sim.step(500)
        peak = max(peak, float(np.max(np.abs(sim.u))))
    assert np.all(np.isfinite(sim.u)) and peak < 1e-6  # Poiseuille flow at g = 2e-9 stays ~2e-7


def test_fused_order_feeds_a_period_two_mode_at_dt1(oracle_mod):
    O = oracle_mod
    sim = _sim(O, False, g=(0.0, 0.0, 0.0))
    sim.step(20)  # linear growth phase (about x100 per 10 steps)
    a = sim.u.copy()
    sim.step(1)
    b = sim.u.copy()
    sim.step(1)
    c = sim.u.copy()
    # consecutive steps are almost exact negatives, and the mode grows
    assert np.sum(a * b) / np.sqrt(np.sum(a * a) * np.sum(b * b)) < -0.99
    assert np.linalg.norm(c) > np.linalg.norm(a)
    spec = np.abs(np.fft.fftn(b.reshape(3, 16, 8, 8)[2]))
    kz, ky, kx = np.unravel_index(np.argmax(spec), spec.shape)
    assert (ky % 4, kx % 4) == (2, 2)  # k_x, k_y = +-pi/2 (z is bounded by the plates)
    while np.max(np.abs(sim.u)) < 1e-3 and sim.s < 2000:
        sim.step(100)
    assert not np.max(np.abs(sim.u)) < 1e-3  # diverged (or NaN)
