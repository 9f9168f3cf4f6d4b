"""Pins of the oracle's lattice-Boltzmann part (Sec. II.C of arXiv:2503.06610).

Each test fixes the oracle against something other than itself: the printed
lattice constants, exact moment identities of the D3Q19 quadrature, the closed
form of a uniformly forced periodic fluid, the textbook Poiseuille profile
between half-way bounce-back plates, shear-wave decay at the viscosity
nu = c_s^2 (tau - 1/2), and mass conservation.
"""
import math
import os

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lattice():
    rows = {}
    cs2 = None
    for line in open(os.path.join(GOLDEN, "d3q19_lattice.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        if k == "cs2":
            cs2 = float(v[0])
        else:
            rows[int(k)] = (int(v[0]), float(v[1]))
    return cs2, rows


def test_lattice_matches_printed_constants(oracle_mod):
    e, w, opp = oracle_mod.lattice()
    cs2, rows = _golden_lattice()
    e2 = np.sum(e * e, axis=1)
    for k, (count, weight) in rows.items():
        assert np.sum(e2 == k) == count
        assert np.allclose(w[e2 == k], weight, rtol=0, atol=1e-16)
    assert len({tuple(v) for v in e}) == 19
    for i in range(19):
        assert np.array_equal(e[opp[i]], -e[i])
    # quadrature identities that make the 2nd-order equilibrium exact
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ e, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), cs2 * np.eye(3), atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(3)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-16)


@pytest.mark.parametrize("shifted", [False, True])
def test_equilibrium_moments(oracle_mod, shifted):
    e, w, _ = oracle_mod.lattice()
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = 1.0 + 0.1 * rng.uniform(-1, 1)
        u = 0.05 * rng.uniform(-1, 1, 3)
        f = oracle_mod.feq(rho, u, shifted)
        full = f + w if shifted else f
        assert abs(full.sum() - rho) < 1e-15
        assert np.allclose(e.T @ full, rho * u, atol=1e-16)
        P = np.einsum("i,ia,ib->ab", full, e, e)
        assert np.allclose(P, rho / 3.0 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
        if shifted:
            assert np.allclose(f, oracle_mod.feq(rho, u, False) - w, atol=1e-16)


def test_guo_source_moments(oracle_mod):
    e, _, _ = oracle_mod.lattice()
    rng = np.random.default_rng(2)
    for _ in range(5):
        u = 0.05 * rng.uniform(-1, 1, 3)
        F = 1e-3 * rng.uniform(-1, 1, 3)
        S = oracle_mod.guo_source(u, F)
        assert abs(S.sum()) < 1e-18
        assert np.allclose(e.T @ S, F, atol=1e-18)
        assert np.allclose(np.einsum("i,ia,ib->ab", S, e, e), np.outer(u, F) + np.outer(F, u), atol=1e-18)


@pytest.mark.parametrize("shifted", [False, True])
def test_uniform_force_periodic_closed_form(oracle_mod, shifted):
    """Fully periodic fluid under a uniform force: with Guo forcing the momentum
    grows by exactly F per step and the moment u of step s is (s - 1/2) g."""
    g = np.array([1e-6, -2e-7, 5e-7])
    p = oracle_mod.OracleParams(nx=4, ny=3, nz=5, walls_z=False, shifted=shifted, tau=0.8, g=tuple(g))
    sim = oracle_mod.OracleSim(p, I.uniform_director(4, 3, 5))
    for s in range(1, 21):
        sim.step(1)
        assert np.allclose(sim.u, ((s - 0.5) * g)[:, None], rtol=1e-9, atol=0)
        assert np.allclose(sim.rho, 1.0, atol=1e-15)
    assert abs(sim.mass() - p.N) < 1e-12 * p.N


def test_poiseuille_exact_at_magic_tau(oracle_mod):
    """Half-way bounce-back with BGK is exact for Poiseuille flow at
    (tau - 1/2)^2 = 3/16; the steady profile is g/(2 nu) (z+1/2)(H-1/2-z) with
    the walls half-way outside the first and last fluid layers."""
    H, gx = 16, 1e-6
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    p = oracle_mod.OracleParams(nx=2, ny=2, nz=H, tau=tau, g=(gx, 0, 0))
    sim = oracle_mod.OracleSim(p, I.uniform_director(2, 2, H)).step(6000)
    z = np.arange(H)
    ua = gx / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
    ux = sim.u[0].reshape(H, 2, 2)
    for j in range(2):
        for i in range(2):
            assert np.max(np.abs(ux[:, j, i] - ua)) <= 1e-10 * ua.max()
    assert np.max(np.abs(sim.u[1:])) < 1e-14 * ua.max()


def test_poiseuille_generic_tau(oracle_mod):
    """At tau = 1: interior nodes satisfy the discrete momentum balance
    nu (u_{z+1} - 2 u_z + u_{z-1}) = -g, the profile is symmetric, and the wall
    slip error stays O(1/H^2) relative."""
    gx = 1e-6
    tau = 1.0
    nu = (tau - 0.5) / 3.0
    errs = []
    for H in (8, 16):
        p = oracle_mod.OracleParams(nx=1, ny=1, nz=H, tau=tau, g=(gx, 0, 0))
        sim = oracle_mod.OracleSim(p, I.uniform_director(1, 1, H)).step(int(40 * H * H))
        ux = sim.u[0]
        curv = nu * (ux[2:] - 2 * ux[1:-1] + ux[:-2]) + gx
        assert np.max(np.abs(curv)) < 1e-10 * gx
        assert np.max(np.abs(ux - ux[::-1])) < 1e-12 * ux.max()
        z = np.arange(H)
        ua = gx / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
        errs.append(np.max(np.abs(ux - ua)) / ua.max())
    assert errs[0] > 0
    assert 3.5 < errs[0] / errs[1] < 4.5   # second order in H


def test_shear_wave_decay_rate(oracle_mod):
    """u_x = U sin(k z) in a periodic box decays as exp(-nu k^2 t) with
    nu = c_s^2 (tau - 1/2), up to the O(k^2) lattice correction."""
    L, U = 64, 1e-4
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / L
    p = oracle_mod.OracleParams(nx=1, ny=1, nz=L, walls_z=False, tau=tau)
    u0 = I.shear_wave(1, 1, L, U)
    sim = oracle_mod.OracleSim(p, I.uniform_director(1, 1, L), u=u0)
    sim.step(100)
    a1 = np.sum(sim.u[0] * np.sin(k * np.arange(L))) * 2 / L
    sim.step(400)
    a2 = np.sum(sim.u[0] * np.sin(k * np.arange(L))) * 2 / L
    rate = -math.log(a2 / a1) / 400
    assert abs(rate / (nu * k * k) - 1.0) < 5e-3


@pytest.mark.parametrize("shifted", [False, True])
def test_mass_conserved_with_walls(oracle_mod, shifted):
    params, n0 = I.tiny_channel(shifted=shifted)
    params = dict(params, nx=8, ny=8, nz=6)
    n0 = I.tilted_director(8, 8, 6, seed=0)
    p = oracle_mod.OracleParams.from_dict(params)
    sim = oracle_mod.OracleSim(p, n0)
    m0 = sim.mass()
    for _ in range(20):
        sim.step(5)
        assert abs(sim.mass() - m0) <= 1e-12 * p.N


def test_shifted_equals_unshifted_in_fp64(oracle_mod):
    """In double precision the shifted store gives essentially the same flow as
    the plain one (Sec. III.A); here the difference is pure round-off."""
    params, _ = I.tiny_channel()
    params = dict(params, nx=8, ny=8, nz=8)
    n0 = I.tilted_director(8, 8, 8, seed=0)
    a = oracle_mod.OracleSim(oracle_mod.OracleParams.from_dict(dict(params, shifted=True)), n0).step(60)
    b = oracle_mod.OracleSim(oracle_mod.OracleParams.from_dict(dict(params, shifted=False)), n0).step(60)
    assert oracle_mod.rel_l2(b.u, a.u) < 1e-9
    assert oracle_mod.rel_l2(b.n, a.n) < 1e-13


@pytest.mark.parametrize("shifted", [False, True])
def test_half_force_shift_closed_form(oracle_mod, shifted):
    """u shifted by H/2 and a Guo source with force F: from the moments of f^eq
    and of S (sum e S = F), the post-collision momentum of a uniform state is
    m + F + (H - F) / (2 tau), and the mass is unchanged."""
    O = oracle_mod
    p = O.OracleParams(nx=4, ny=3, nz=2, walls_z=False, shifted=shifted, tau=0.7)
    N = p.N
    rho0, u0 = 1.03, np.array([2e-3, -1e-3, 5e-4])
    f = O.init_populations(p, np.full(N, rho0), np.tile(u0[:, None], (1, N)))
    e, _, _ = O.lattice()
    m = e.T @ f[:, 0]
    H, F = np.array([3e-4, -2e-4, 1e-4]), np.array([-1e-4, 4e-4, 2e-4])
    fn, rho, u = O.lb_step(p, f, np.tile(F[:, None], (1, N)), Fu=np.tile(H[:, None], (1, N)))
    m_new = e.T @ fn
    expect = m + F + (H - F) / (2 * p.tau)
    assert np.max(np.abs(m_new - expect[:, None])) < 1e-15
    assert np.allclose(u[:, 0], (m + H / 2) / rho0, rtol=0, atol=1e-16)
    assert abs(np.sum(fn) - np.sum(f)) < 1e-13


def _push_paper_loop(O, p, n0, steps):
    """The loop of Sec. II.D in the printed order, written independently of the
    oracle's LB step: push streaming by array shifts on a periodic lattice,
    macroscopic fields with the force in effect, the FD update and force when
    due, then the collision (Eq. shifted-lbe with Guo's source).  The lattice
    is the set of integer vectors with |e|^2 <= 2 and the printed weights; the
    FD update and the force come from the oracle (pinned separately)."""
    cs2, rows = _golden_lattice()
    e, _, _ = O.lattice()           # the oracle's population order, checked against the golden file
    w = np.array([rows[int(v @ v)][1] for v in e])
    nz, ny, nx = p.nz, p.ny, p.nx
    N = p.N
    f = O.init_populations(p, np.ones(N), np.zeros((3, N)))
    n = np.asarray(n0, dtype=np.float64).reshape(3, N).copy()
    u = np.zeros((3, N))
    F = O.force(p, O.stress(p, n, u))
    g = np.array(p.g)[:, None]
    for s in range(1, steps + 1):
        fs = f.reshape(19, nz, ny, nx)
        f = np.stack([np.roll(fs[i], shift=(e[i, 2], e[i, 1], e[i, 0]), axis=(0, 1, 2)) for i in range(19)])
        f = f.reshape(19, N)
        sm = f.sum(axis=0)
        rho = 1.0 + sm if p.shifted else sm
        Ft = F + rho * g
        u = (e.T @ f + 0.5 * Ft) / rho
        if s % p.dt_fd == 0:
            n = O.fd_step(p, n, u)
            F = O.force(p, O.stress(p, n, u))
            Ft = F + rho * g
        eu = e @ u
        uu = np.sum(u * u, axis=0)
        feq = w[:, None] * rho * (1 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - uu / (2 * cs2))
        if p.shifted:
            feq = feq - w[:, None]
        eF = e @ Ft
        uF = np.sum(u * Ft, axis=0)
        S = w[:, None] * (eF / cs2 + (eu * eF) / cs2 ** 2 - uF / cs2)
        f = f - (f - feq) / p.tau + (1 - 1 / (2 * p.tau)) * S
    return f, n, u


@pytest.mark.parametrize("dt_fd", [1, 3])
def test_paper_order_matches_push_form_loop(oracle_mod, dt_fd):
    O = oracle_mod
    d = dict(nx=10, ny=8, nz=6, walls_z=False, shifted=True, tau=0.8, g=(2e-5, 0.0, -1e-5), K=0.02,
             q0=2 * math.pi / 8, gamma1=1.0, gamma2=-0.9, alpha1=0.01, alpha2=-0.95, alpha3=0.05,
             alpha4p=0.02, alpha5=0.45, alpha6=-0.45, W0=0.003, dt_fd=dt_fd)
    n0 = I.skyrmion_tubes(10, 8, 6, [(5.0, 4.0)], 3.0)
    p = O.OracleParams(paper_order=True, **d)
    steps = 7
    f_ref, n_ref, u_ref = _push_paper_loop(O, p, n0, steps)
    sim = O.OracleSim(p, n0).step(steps)
    assert np.max(np.abs(sim.f - f_ref)) < 1e-14
    assert np.max(np.abs(sim.n - n_ref)) < 1e-14
    # the fused order (collision before the FD update) differs: the check discriminates
    other = O.OracleSim(O.OracleParams(paper_order=False, **d), n0).step(steps)
    assert np.max(np.abs(other.f - f_ref)) > 1e-9
