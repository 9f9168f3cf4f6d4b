"""Pins of the oracle's director / stress part (Secs. II.A-II.B of arXiv:2503.06610).

* the molecular field h is minus the gradient of the lattice Frank energy
  (brute-force finite differences on tiny grids, periodic and with walls);
* a small twist mode decays as the Heun amplification factor of the discrete
  Laplacian predicts, and as exp(-K k^2 t / gamma1) in the continuum limit;
* the uniform and the helical ground states are stationary;
* the Frank energy does not increase at rest; |n| = 1 after every step;
* the elastic stress is -d_a n_g df/d(d_b n_g), checked by differentiating the
  one-constant energy density numerically;
* the symmetric part of the viscous stress is the derivative of the
  Ericksen-Leslie dissipation function, its antisymmetric part balances the
  molecular-field torque, and N agrees with the director equation;
* the force is the divergence over the second stress index, with zero ghost
  stress beyond the plates;
* the alpha_4' term adds alpha_4'/2 to the kinematic viscosity of a shear wave.
"""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

LESLIE = I.LESLIE_ALIGN_09


def _grad_energy(O, p, n, d=1e-6):
    g = np.zeros_like(n)
    for a in range(3):
        for s in range(p.N):
            npl = n.copy()
            npl[a, s] += d
            nm = n.copy()
            nm[a, s] -= d
            g[a, s] = (O.frank_energy(p, npl) - O.frank_energy(p, nm)) / (2 * d)
    return g


@pytest.mark.parametrize("walls,anchoring,nz", [(False, "homeotropic", 4), (True, "homeotropic", 4),
                                                (True, "none", 4), (True, "none", 1), (True, "none", 2)])
def test_molecular_field_is_energy_gradient(oracle_mod, walls, anchoring, nz):
    """h = -dE_d/dn at every site (Sec. II.A), plate layers included.  Without
    anchoring the plates carry no link energy (a free surface), so the chiral
    term at the two plate layers lacks its link to the ghost layer; a central
    curl over copied ghosts would add a spurious tangential torque K q0 (z x n)
    there, which this comparison rejects (q0 and W0 are nonzero)."""
    O = oracle_mod
    p = O.OracleParams(nx=4, ny=3, nz=nz, walls_z=walls, anchoring=anchoring, K=0.7, q0=0.9, W0=0.3)
    n = I.random_director(4, 3, nz, seed=3)
    h = O.molecular_field(p, n)
    g = _grad_energy(O, p, n)
    assert np.max(np.abs(g + h)) < 1e-7 * np.max(np.abs(h))


def test_twist_mode_decay(oracle_mod):
    O = oracle_mod
    nx, K, g1, dt, eps, m = 32, 0.04, 1.0, 2, 1e-3, 50
    p = O.OracleParams(nx=nx, ny=2, nz=2, walls_z=False, K=K, gamma1=g1, dt_fd=dt)
    n = I.twist_mode(nx, 2, 2, eps)
    u = np.zeros((3, p.N))
    for _ in range(m):
        n = O.fd_step(p, n, u)
    k = 2 * math.pi / nx
    x = np.arange(nx)
    theta = np.arctan2(n[2], n[1]).reshape(2, 2, nx)
    lam = K / g1 * (2 - 2 * math.cos(k))
    heun = eps * (1 - lam * dt + 0.5 * (lam * dt) ** 2) ** m
    cont = eps * math.exp(-K * k * k * m * dt / g1)
    for j in range(2):
        for i in range(2):
            amp = np.sum(theta[j, i] * np.sin(k * x)) * 2 / nx
            assert abs(amp / heun - 1) < 1e-6          # O(eps^2) from the nonlinearity
            assert abs(amp / cont - 1) < 2e-3          # lattice O(k^2) + O(dt^2) corrections
    assert np.max(np.abs(np.linalg.norm(n, axis=0) - 1)) < 1e-14


def test_helix_ground_state_is_stationary(oracle_mod):
    O = oracle_mod
    q = 2 * math.pi / 16
    p = O.OracleParams(nx=4, ny=4, nz=16, walls_z=False, tau=1.0, K=0.04, q0=q, **LESLIE)
    n0 = I.helix(4, 4, 16, q)
    sim = O.OracleSim(p, n0).step(1000)
    assert np.max(np.abs(sim.n - n0)) < 1e-14
    assert np.max(np.abs(sim.u)) < 1e-15


def test_uniform_homeotropic_channel_is_stationary(oracle_mod):
    O = oracle_mod
    p = O.OracleParams(nx=4, ny=4, nz=8, walls_z=True, tau=1.0, K=0.04, q0=0.0, **LESLIE)
    n0 = I.uniform_director(4, 4, 8)
    sim = O.OracleSim(p, n0).step(500)
    assert np.max(np.abs(sim.n - n0)) == 0.0
    assert np.max(np.abs(sim.u)) == 0.0


@pytest.mark.parametrize("q0,anchoring,W0", [(0.0, "homeotropic", 0.0), (2 * math.pi / 8, "homeotropic", 0.0),
                                            (2 * math.pi / 8, "none", 0.0), (2 * math.pi / 8, "none", 0.01)])
def test_energy_non_increasing_at_rest(oracle_mod, q0, anchoring, W0):
    """At rest the director equation is the gradient flow of E_d: E_d does not
    increase, plates without anchoring (and the bulk W0 term) included."""
    O = oracle_mod
    p = O.OracleParams(nx=8, ny=8, nz=6, walls_z=True, anchoring=anchoring, K=0.04, q0=q0, W0=W0, gamma1=1.0,
                       dt_fd=2)
    n = I.tilted_director(8, 8, 6, amplitude=0.5, seed=4)
    u = np.zeros((3, p.N))
    E = [O.frank_energy(p, n)]
    for _ in range(40):
        n = O.fd_step(p, n, u)
        E.append(O.frank_energy(p, n))
        assert np.max(np.abs(np.linalg.norm(n, axis=0) - 1)) < 1e-14
    dE = np.diff(E)
    assert np.all(dE <= 1e-14 * abs(E[0]))
    assert E[-1] < E[0]


def _energy_density(K, q0, n, G):
    """One-constant chiral density f = K/2 G:G + K q0 n.curl + K q0^2/2, G[b,g] = d_b n_g."""
    curl = np.array([G[1, 2] - G[2, 1], G[2, 0] - G[0, 2], G[0, 1] - G[1, 0]])
    return 0.5 * K * np.sum(G * G) + K * q0 * n @ curl + 0.5 * K * q0 * q0


def test_elastic_stress_is_energy_derivative(oracle_mod):
    O = oracle_mod
    K, q0 = 0.37, 1.3
    p = O.OracleParams(nx=1, ny=1, nz=1, K=K, q0=q0)
    rng = np.random.default_rng(5)
    for _ in range(5):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        G = rng.normal(size=(3, 3))
        dfdG = np.zeros((3, 3))
        d = 1e-6
        for b in range(3):
            for g in range(3):
                Gp = G.copy()
                Gp[b, g] += d
                Gm = G.copy()
                Gm[b, g] -= d
                dfdG[b, g] = (_energy_density(K, q0, n, Gp) - _energy_density(K, q0, n, Gm)) / (2 * d)
        expect = -np.einsum("ag,bg->ab", G, dfdG)
        assert np.allclose(O.elastic_stress_point(p, n, G), expect, atol=1e-8)


def _dissipation(al, g1, g2, n, D, N):
    """Ericksen-Leslie dissipation function 2R(D, N) (Parodi relation assumed)."""
    Dn = D @ n
    nDn = n @ Dn
    return 0.5 * (al[0] * nDn ** 2 + 2 * g2 * N @ Dn + al[3] * np.sum(D * D)
                  + (al[4] + al[5]) * Dn @ Dn + g1 * N @ N)


def test_viscous_stress_from_dissipation_and_torque(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(6)
    a1, a2, a3, a4, a5, a6 = 0.0373, -0.4496, -0.0203, 0.9318, 0.3084, -0.1617
    g1, g2 = a3 - a2, a3 + a2
    a6 = g2 + a5                                   # enforce Parodi exactly
    p = O.OracleParams(nx=1, ny=1, nz=1, alpha1=a1, alpha2=a2, alpha3=a3, alpha4p=a4, alpha5=a5,
                       alpha6=a6, gamma1=g1, gamma2=g2)
    al = (a1, a2, a3, a4, a5, a6)
    for _ in range(5):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        A = rng.normal(size=(3, 3))
        D = 0.5 * (A + A.T)
        h = rng.normal(size=3)
        Nv = O.transport_point(n, h, D, g1, g2)
        sig = O.viscous_stress_point(p, n, D, Nv)
        # symmetric part = dR/dD at fixed N (symmetrised derivative)
        dRdD = np.zeros((3, 3))
        d = 1e-6
        for i in range(3):
            for j in range(3):
                E = np.zeros((3, 3))
                E[i, j] += 0.5 * d
                E[j, i] += 0.5 * d
                dRdD[i, j] = (_dissipation(al, g1, g2, n, D + E, Nv) - _dissipation(al, g1, g2, n, D - E, Nv)) / (2 * d)
        assert np.allclose(0.5 * (sig + sig.T), dRdD, atol=1e-8)
        # antisymmetric part balances the torque of h_perp
        hp = h - (h @ n) * n
        assert np.allclose(0.5 * (sig - sig.T), -0.5 * (np.outer(hp, n) - np.outer(n, hp)), atol=1e-12)
        assert abs(Nv @ n) < 1e-14


def test_transport_matches_director_equation(oracle_mod):
    """N = dn/dt + u.grad n - W n with dn/dt from the director equation,
    projected normal to n, equals the transport used in the stress."""
    O = oracle_mod
    p = O.OracleParams(nx=5, ny=4, nz=3, walls_z=False, K=0.2, q0=0.7, W0=0.1, **LESLIE)
    n = I.random_director(5, 4, 3, seed=7)
    u = I.random_velocity(5, 4, 3, 1e-2, seed=8)
    ndot = O.director_rate(p, n, u)
    h = O.molecular_field(p, n)
    N3 = n.reshape(3, 3, 4, 5)
    U3 = u.reshape(3, 3, 4, 5)

    def cd(f, axis):  # central difference on the periodic grid, axis in (x,y,z)
        ax = {0: 3, 1: 2, 2: 1}[axis]
        return 0.5 * (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax))

    grad_n = np.stack([cd(N3, b) for b in range(3)])        # [b][c] = d_b n_c
    grad_u = np.stack([cd(U3, b) for b in range(3)])        # [a][m] = d_a u_m
    for s in range(0, p.N, 7):
        z, y, x = np.unravel_index(s, (3, 4, 5))
        nn = n[:, s]
        du = grad_u[:, :, z, y, x]
        D = 0.5 * (du + du.T)
        W = 0.5 * (du.T - du)                               # W[m][g] = 1/2 (d_g u_m - d_m u_g)
        adv = u[:, s] @ grad_n[:, :, z, y, x]
        Nfull = ndot[:, s] + adv - W @ nn
        Nperp = Nfull - (Nfull @ nn) * nn
        Nv = O.transport_point(nn, h[:, s], D, p.gamma1, p.gamma2)
        assert np.allclose(Nv, Nperp, atol=1e-13)


@pytest.mark.parametrize("walls", [False, True])
def test_force_is_divergence_over_second_index(oracle_mod, walls):
    O = oracle_mod
    nx, ny, nz = 4, 3, 8
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=walls)
    k = 2 * math.pi / nz
    z = np.repeat(np.arange(nz), nx * ny).astype(float)
    sigma = np.zeros((9, p.N))
    sigma[0 * 3 + 2] = np.sin(k * z)        # sigma_xz(z)
    sigma[2 * 3 + 0] = 5.0                  # sigma_zx uniform -> no force
    F = O.force(p, sigma)
    expect = math.sin(k) * np.cos(k * z)    # exact central difference of sin(kz)
    if walls:
        top = z == nz - 1
        bot = z == 0
        expect = np.where(bot, 0.5 * np.sin(k * (z + 1)), expect)
        expect = np.where(top, -0.5 * np.sin(k * (z - 1)), expect)
    assert np.allclose(F[0], expect, atol=1e-15)
    assert np.allclose(F[1], 0.0, atol=0)
    if walls:
        # uniform sigma_zx still has no x- or y-gradient; at the plates the
        # ghost stress is zero, but only d_z sigma_az enters F_a.
        assert np.allclose(F[2], 0.0, atol=0)
    else:
        assert np.allclose(F[2], 0.0, atol=0)


def test_alpha4p_adds_viscosity(oracle_mod):
    """With only alpha_4' non-zero the LC stress is alpha_4' D, and a shear wave
    decays at nu + alpha_4'/2 (central-of-central: k^2 -> sin^2 k)."""
    O = oracle_mod
    L, U, tau, a4p = 32, 1e-4, 0.8, 0.1
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / L
    p = O.OracleParams(nx=1, ny=1, nz=L, walls_z=False, tau=tau, alpha4p=a4p, gamma1=1.0, dt_fd=1)
    u0 = I.shear_wave(1, 1, L, U)
    sim = O.OracleSim(p, I.uniform_director(1, 1, L, (1, 0, 0)), u=u0)
    sim.step(50)
    zz = np.arange(L)
    a1 = np.sum(sim.u[0] * np.sin(k * zz)) * 2 / L
    sim.step(200)
    a2 = np.sum(sim.u[0] * np.sin(k * zz)) * 2 / L
    rate = -math.log(a2 / a1) / 200
    expect = nu * k * k + 0.5 * a4p * math.sin(k) ** 2
    assert abs(rate / expect - 1) < 1e-2
    # and the LB-only rate would be clearly different
    assert abs(nu * k * k / expect - 1) > 0.3


def test_unit_norm_after_coupled_steps(oracle_mod):
    O = oracle_mod
    params, _ = I.tiny_channel()
    params = dict(params, nx=8, ny=8, nz=6)
    n0 = I.tilted_director(8, 8, 6, seed=1)
    sim = O.OracleSim(O.OracleParams.from_dict(params), n0).step(30)
    assert np.max(np.abs(np.linalg.norm(sim.n, axis=0) - 1)) < 1e-14


def test_centroid_recovers_tube_centre(oracle_mod):
    O = oracle_mod
    nx, ny, nz = 40, 36, 4
    p = O.OracleParams(nx=nx, ny=ny, nz=nz)
    for c in [(20.0, 18.0), (1.0, 35.0)]:     # second one wraps around the periodic edges
        n = I.skyrmion_tubes(nx, ny, nz, [c], 8.0)
        got = O.centroids(p, n, [c])[0]
        d = (got - np.array(c) + 0.5 * np.array([nx, ny])) % np.array([nx, ny]) - 0.5 * np.array([nx, ny])
        assert np.max(np.abs(d)) < 1e-9


def test_paper_table_parodi_relation():
    """Table I of the paper satisfies Parodi's relation alpha6 - alpha5 = alpha2 + alpha3
    to the printed precision, supporting the reading gamma2 = alpha2 + alpha3."""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_mbba.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    assert abs((vals["alpha6"] - vals["alpha5"]) - (vals["alpha2"] + vals["alpha3"])) < 5e-4


# ------------------------------------------------------------------ three-constant Frank energy

K3 = dict(K=0.01, K11=0.02, K22=0.005, K33=0.03)


def test_frank3_closed_form_energies(oracle_mod):
    """Delta f of a helix (pure twist: div = 0, w = -sin(q) n) and of a
    splay-bend wave n = (sin kx, 0, cos kx) (n.w = 0) in closed form, with the
    central-difference factors sin q, sin k."""
    O = oracle_mod
    q0 = 0.3
    nz, q = 16, 2 * math.pi / 16
    p = O.OracleParams(nx=2, ny=3, nz=nz, walls_z=False, q0=q0, **K3)
    E, _ = O.frank3_field(p, I.helix(2, 3, nz, q))
    assert abs(E - p.N * 0.5 * (p.K22 - p.K) * (q0 - math.sin(q)) ** 2) < 1e-15 * p.N
    nx, k = 12, 2 * math.pi / 12
    p = O.OracleParams(nx=nx, ny=2, nz=3, walls_z=False, q0=q0, **K3)
    x = np.arange(nx)
    n = np.zeros((3, 3, 2, nx))
    n[0] = np.sin(k * x)
    n[2] = np.cos(k * x)
    E, _ = O.frank3_field(p, n.reshape(3, -1))
    per_col = np.sum(0.5 * (p.K11 - p.K) * np.cos(k * x) ** 2 * math.sin(k) ** 2
                     + 0.5 * (p.K22 - p.K) * q0 ** 2
                     + 0.5 * (p.K33 - p.K) * np.sin(k * x) ** 2 * math.sin(k) ** 2)
    assert abs(E - 6 * per_col) < 1e-15 * p.N


def test_frank3_point_derivatives(oracle_mod):
    """d Delta f / dn and d Delta f / d(d_b n_c) against central differences of Delta f."""
    O = oracle_mod
    p = O.OracleParams(nx=2, ny=2, nz=2, q0=0.4, **K3)
    rng = np.random.default_rng(4)
    for _ in range(5):
        n3 = rng.normal(size=3)
        G = 0.3 * rng.normal(size=(3, 3))
        _, dfdn, P = O.frank3_point(p, n3, G)
        d = 1e-6
        for c in range(3):
            e = np.zeros(3)
            e[c] = d
            num = (O.frank3_point(p, n3 + e, G)[0] - O.frank3_point(p, n3 - e, G)[0]) / (2 * d)
            assert abs(num - dfdn[c]) < 1e-9
        for b in range(3):
            for c in range(3):
                E = np.zeros((3, 3))
                E[b, c] = d
                num = (O.frank3_point(p, n3, G + E)[0] - O.frank3_point(p, n3, G - E)[0]) / (2 * d)
                assert abs(num - P[b, c]) < 1e-9


@pytest.mark.parametrize("walls", [False, True])
def test_frank3_field_is_energy_gradient(oracle_mod, walls):
    """Full h (one-constant part + correction) = -dE_d/dn, periodic and with
    homeotropic plates."""
    O = oracle_mod
    p = O.OracleParams(nx=4, ny=3, nz=4, walls_z=walls, anchoring="homeotropic", q0=0.9, W0=0.3,
                       K=0.7, K11=1.1, K22=0.4, K33=1.6)
    n = I.random_director(4, 3, 4, seed=5)
    h = O.molecular_field(p, n)
    g = _grad_energy(O, p, n)
    assert np.max(np.abs(g + h)) < 1e-7 * np.max(np.abs(h))


@pytest.mark.parametrize("anchoring", ["none", "homeotropic"])
def test_frank3_correction_field_with_plates(oracle_mod, anchoring):
    """The correction's field is -d(sum Delta f)/dn also when the ghost layer
    copies the adjacent fluid layer (no anchoring): the copy's dependence on
    that layer is part of the derivative."""
    O = oracle_mod
    p = O.OracleParams(nx=4, ny=3, nz=4, walls_z=True, anchoring=anchoring, q0=0.9, K=0.7, K11=1.1, K22=0.4,
                       K33=1.6)
    n = I.random_director(4, 3, 4, seed=6)
    _, hd = O.frank3_field(p, n)
    d = 1e-6
    g = np.zeros_like(hd)
    for a in range(3):
        for s_ in range(p.N):
            npl = n.copy()
            npl[a, s_] += d
            nm = n.copy()
            nm[a, s_] -= d
            g[a, s_] = (O.frank3_field(p, npl)[0] - O.frank3_field(p, nm)[0]) / (2 * d)
    assert np.max(np.abs(g + hd)) < 1e-7 * np.max(np.abs(hd))


def test_frank3_equal_constants_reduce_to_one_constant(oracle_mod):
    O = oracle_mod
    d = dict(nx=6, ny=5, nz=4, walls_z=True, K=0.02, q0=0.5, W0=0.01, tau=0.8, g=(1e-5, 0, 0), **LESLIE)
    n0 = I.skyrmion_tubes(6, 5, 4, [(3.0, 2.5)], 2.0)
    a = O.OracleSim(O.OracleParams(**d), n0).step(5)
    b = O.OracleSim(O.OracleParams(K11=0.02, K22=0.02, K33=0.02, **d), n0).step(5)
    assert np.array_equal(a.n, b.n) and np.array_equal(a.f, b.f)


@pytest.mark.parametrize("axis,Kii", [(0, "K11"), (1, "K22"), (2, "K33")])
def test_frank3_splay_twist_bend_decay(oracle_mod, axis, Kii):
    """A small tilt dn_x = eps sin(k r_axis) of n = z_hat is a pure splay (along
    x), twist (along y) or bend (along z) mode.  It decays at the discrete rate
    lambda = [2 K (1 - cos k) + (K_ii - K) sin^2 k] / gamma1 (compact one-constant
    part plus the central-difference correction), i.e. by the Heun factor per step."""
    O = oracle_mod
    L, g1, dt, eps, m = 8, 1.0, 5, 1e-6, 20
    dims = [2, 2, 2]
    dims[axis] = L
    p = O.OracleParams(nx=dims[0], ny=dims[1], nz=dims[2], walls_z=False, gamma1=g1, dt_fd=dt, **K3)
    k = 2 * math.pi / L
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    r = (x, y, z)[axis]
    n = np.zeros((3,) + x.shape)
    n[0] = eps * np.sin(k * r)
    n[2] = 1.0
    n = (n / np.linalg.norm(n, axis=0)).reshape(3, -1)
    u = np.zeros((3, p.N))
    for _ in range(m):
        n = O.fd_step(p, n, u)
    lam = (2 * p.K * (1 - math.cos(k)) + (getattr(p, Kii) - p.K) * math.sin(k) ** 2) / g1
    heun = eps * (1 - lam * dt + 0.5 * (lam * dt) ** 2) ** m
    rr = r.reshape(-1)
    amp = np.sum(n[0] * np.sin(k * rr)) * 2 / rr.size
    assert abs(amp / heun - 1) < 1e-6


def test_flow_alignment_leslie_angle(oracle_mod):
    """Without elasticity (K = 0) every site evolves on its own under the local
    shear: for n = (sin t, 0, cos t) in u_x(z), the director equation gives
    dt/dt = (g/2)(1 - lambda cos 2t), lambda = gamma2/gamma1, g = du_x/dz.  A
    flow-aligning nematic (|lambda| > 1) settles at cos 2t = 1/lambda, with
    sin 2t of the sign opposite to lambda g (the stable root) -- the Leslie angle.
    The Heun map has the same fixed point, so the angle is exact."""
    O = oracle_mod
    nz = 16
    lam = -1.5
    p = O.OracleParams(nx=1, ny=1, nz=nz, walls_z=False, K=0.0, gamma1=1.0, gamma2=lam, dt_fd=1)
    z = np.arange(nz)
    k = 2 * math.pi / nz
    u = np.zeros((3, nz))
    u[0] = 0.05 * np.sin(k * z)
    n = np.zeros((3, nz))
    n[0] = n[2] = math.sqrt(0.5)
    for _ in range(6000):
        n = O.fd_step(p, n, u)
    shear = 0.5 * (np.roll(u[0], -1) - np.roll(u[0], 1))   # central du_x/dz of the oracle
    t = np.arctan2(n[0], n[2])
    for zz in range(nz):
        if abs(shear[zz]) < 1e-12:
            continue
        c2, s2 = math.cos(2 * t[zz]), math.sin(2 * t[zz])
        assert abs(c2 - 1 / lam) < 1e-9, zz
        assert s2 * lam * shear[zz] < 0, zz
    assert np.max(np.abs(n[1])) < 1e-15


def test_effective_shear_viscosity_at_rest_director(oracle_mod):
    """Assembled stress under shear u_x(z) with a director that the director
    equation leaves at rest (K = 0): at the Leslie angle (n = (sin t, 0, cos t),
    cos 2t = gamma1/gamma2) and along the vorticity axis (n = y_hat), N = -W n, and
    the shear stress is the effective viscosity of a held director (de Gennes &
    Prost, Sec. 5.1) times the local rate g = du_x/dz:
        eta(t) = a1 sin^2 t cos^2 t + [a4' + (a5 - a2) cos^2 t + (a3 + a6) sin^2 t] / 2,
        eta(y_hat) = a4' / 2,
    with sigma_xz = sigma_zx (no torque).  Swapping a2 with a3 or a5 with a6, a
    transposed strain or vorticity, or a wrong coupling gamma2/gamma1 in N breaks it."""
    O = oracle_mod
    nz = 16
    a = dict(alpha1=0.3, alpha2=-1.25, alpha3=-0.25, alpha4p=0.4, alpha5=1.0, alpha6=-0.5)
    g1, g2 = a["alpha3"] - a["alpha2"], a["alpha3"] + a["alpha2"]   # Parodi: gamma1 = a3 - a2, gamma2 = a6 - a5
    assert abs(g2 - (a["alpha6"] - a["alpha5"])) < 1e-15
    p = O.OracleParams(nx=1, ny=1, nz=nz, walls_z=False, K=0.0, q0=0.0, W0=0.0, gamma1=g1, gamma2=g2, **a)
    z = np.arange(nz)
    u = np.zeros((3, nz))
    u[0] = 0.01 * np.sin(2 * math.pi * z / nz)
    rate = 0.5 * (np.roll(u[0], -1) - np.roll(u[0], 1))   # central du_x/dz
    t = 0.5 * math.acos(g1 / g2)
    s, c = math.sin(t), math.cos(t)
    eta = a["alpha1"] * s * s * c * c + 0.5 * (a["alpha4p"] + (a["alpha5"] - a["alpha2"]) * c * c
                                               + (a["alpha3"] + a["alpha6"]) * s * s)
    for n_vec, eta_ref in (((s, 0.0, c), eta), ((0.0, 1.0, 0.0), 0.5 * a["alpha4p"])):
        n = np.tile(np.asarray(n_vec)[:, None], (1, nz))
        sig = O.stress(p, n, u)
        sxz, szx = sig[3 * 0 + 2], sig[3 * 2 + 0]
        assert np.max(np.abs(sxz - eta_ref * rate)) < 1e-15
        assert np.max(np.abs(szx - eta_ref * rate)) < 1e-15
    # away from a rest state the held-director formula does not apply
    n = np.tile(np.array([math.sin(0.3), 0.0, math.cos(0.3)])[:, None], (1, nz))
    eta03 = a["alpha1"] * math.sin(0.3) ** 2 * math.cos(0.3) ** 2 + 0.5 * (
        a["alpha4p"] + (a["alpha5"] - a["alpha2"]) * math.cos(0.3) ** 2 + (a["alpha3"] + a["alpha6"]) * math.sin(0.3) ** 2)
    assert np.max(np.abs(O.stress(p, n, u)[2] - eta03 * rate)) > 1e-6


def test_frank_energy_closed_forms(oracle_mod):
    """Absolute lattice Frank energy (the diagnostic) of states with a closed
    form.  Helix n = (cos qz, sin qz, 0): every z-link carries
    K/2 |m - n|^2 = K (1 - cos q) and the chiral term -K q0 (n x m)_z = -K q0 sin q,
    so E/N = K (1 - cos q) - K q0 sin q + K q0^2/2 (-> K/2 (q - q0)^2 for small q,
    the continuum cholesteric); without anchoring the two ghost links of a column
    carry nothing.  Uniform z_hat: E/N = K q0^2/2 - W0/2."""
    O = oracle_mod
    K, q0, W0 = 0.02, 0.4, 3e-3
    nx, ny, nz = 3, 2, 12
    for m in (1, 2, -1):
        q = 2 * math.pi * m / nz
        n = I.helix(nx, ny, nz, q)
        link = K * (1 - math.cos(q)) - K * q0 * math.sin(q)
        p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=False, K=K, q0=q0)
        assert abs(O.frank_energy(p, n) - nx * ny * nz * (link + 0.5 * K * q0 ** 2)) < 1e-13
        p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="none", K=K, q0=q0)
        assert abs(O.frank_energy(p, n) - nx * ny * ((nz - 1) * link + nz * 0.5 * K * q0 ** 2)) < 1e-13
    # the right-handed helix (q = q0 > 0) is the lower one
    q = 2 * math.pi / nz
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=False, K=K, q0=q0)
    assert O.frank_energy(p, I.helix(nx, ny, nz, q)) < O.frank_energy(p, I.helix(nx, ny, nz, -q))
    for walls, anch in ((False, "none"), (True, "homeotropic")):
        p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=walls, anchoring=anch, K=K, q0=q0, W0=W0)
        E = O.frank_energy(p, I.uniform_director(nx, ny, nz))
        assert abs(E - nx * ny * nz * (0.5 * K * q0 ** 2 - 0.5 * W0)) < 1e-13
