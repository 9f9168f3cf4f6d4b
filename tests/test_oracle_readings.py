"""Pins of the oracle's reading flags, the choices the paper leaves open.

* renorm_predictor: a director turned by a steady vorticity (K = 0, no flow
  alignment) turns per FD step by the angle of Heun's method applied to a
  rotation: atan2(w dt, 1 - (w dt)^2/2) when only the corrected director is
  renormalised, and atan2(w dt (1 + 1/s)/2, 1 - (w dt)^2/(2 s)), s = sqrt(1 +
  (w dt)^2), when the predictor is renormalised too.
* lap_wide: second derivatives as central differences of central differences
  (Sec. II.B's first-derivative stencil applied twice) turn the decay rate of a
  twist mode from (K/gamma1)(2 - 2 cos k) into (K/gamma1) sin^2 k, so the
  checkerboard mode (k = pi) does not decay at all; between plates without
  anchoring a field that does not depend on z evolves as in a periodic box.
* n_from_rate: N built from the corrector's averaged rate converges to the
  director-equation form as dt_FD -> 0, at first order (a missing projection
  or a wrong sign of u.grad n or W n would leave a difference of order one).
* ghost_sigma: the central divergence telescopes, so the total force over the
  channel is sum_xy [sigma_az(top layer) - sigma_az(bottom layer)] with
  mirrored ghost stress and half of that with zero ghost stress; a uniform
  stress exerts no force with mirrored ghosts.
"""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I


def _angle(n):
    return np.arctan2(n[2], n[0])


@pytest.mark.parametrize("renorm", [False, True])
def test_predictor_renormalisation_rotation_angle(oracle_mod, renorm):
    O = oracle_mod
    L, S, dt, m = 16, 0.3, 4, 7
    p = O.OracleParams(nx=1, ny=1, nz=L, walls_z=False, K=0.0, gamma1=1.0, gamma2=0.0, dt_fd=dt,
                       renorm_predictor=renorm)
    k = 2 * math.pi / L
    z = np.arange(L)
    u = np.zeros((3, L))
    u[0] = S * np.sin(k * z)
    n = np.zeros((3, L))
    n[0] = 1.0
    phi0 = _angle(n)
    for _ in range(m):
        n = O.fd_step(p, n, u)
    # n = (cos phi, 0, sin phi) turns at w = -(d_z u_x)/2 with the central derivative
    a = S * (np.sin(k * (z + 1)) - np.sin(k * (z - 1))) / 2
    wdt = -0.5 * a * dt
    s = np.sqrt(1 + wdt ** 2)
    step = np.arctan2(wdt * (1 + 1 / s) / 2, 1 - wdt ** 2 / (2 * s)) if renorm else np.arctan2(wdt, 1 - wdt ** 2 / 2)
    expect = phi0 + m * step
    assert np.max(np.abs(np.angle(np.exp(1j * (_angle(n) - expect))))) < 1e-12
    other = np.arctan2(wdt, 1 - wdt ** 2 / 2) if renorm else np.arctan2(wdt * (1 + 1 / s) / 2, 1 - wdt ** 2 / (2 * s))
    assert np.max(np.abs(m * (step - other))) > 1e-4  # the two readings are told apart


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("nx", [32, 2])
def test_wide_laplacian_twist_decay(oracle_mod, wide, nx):
    O = oracle_mod
    K, g1, dt, eps, m = 0.04, 1.0, 2, 1e-3, 30
    p = O.OracleParams(nx=nx, ny=2, nz=2, walls_z=False, K=K, gamma1=g1, dt_fd=dt, lap_wide=wide)
    k = 2 * math.pi / nx if nx > 2 else math.pi  # nx = 2: the checkerboard mode
    x = np.arange(nx)
    if nx == 2:
        theta0 = eps * np.cos(k * x)
    else:
        theta0 = eps * np.sin(k * x)
    n = np.stack([np.zeros(nx * 4), np.cos(np.tile(theta0, 4)), np.sin(np.tile(theta0, 4))])
    u = np.zeros((3, p.N))
    for _ in range(m):
        n = O.fd_step(p, n, u)
    lam = K / g1 * (math.sin(k) ** 2 if wide else 2 - 2 * math.cos(k))
    heun = (1 - lam * dt + 0.5 * (lam * dt) ** 2) ** m
    theta = np.arctan2(n[2], n[1]).reshape(2, 2, nx)
    basis = np.cos(k * x) if nx == 2 else np.sin(k * x)
    amp = np.sum(theta * basis, axis=-1) / np.sum(basis * basis) / eps
    assert np.max(np.abs(amp / heun - 1)) < 1e-6
    if nx == 2 and wide:
        assert abs(heun - 1) < 1e-15  # sin^2(pi) = 0: the checkerboard does not decay


def test_wide_laplacian_free_plates_equal_periodic_z(oracle_mod):
    O = oracle_mod
    nx, ny, nz = 12, 4, 5
    n0 = I.twist_mode(nx, ny, nz, amplitude=0.3)
    u = np.zeros((3, nx * ny * nz))
    out = []
    for walls in (False, True):
        p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=walls, anchoring="none", K=0.05, gamma1=1.0, dt_fd=3,
                           lap_wide=True)
        n = n0
        for _ in range(5):
            n = O.fd_step(p, n, u)
        out.append(n)
    assert np.max(np.abs(out[0] - out[1])) < 1e-15
    assert np.max(np.abs(out[0] - n0)) > 1e-3


def test_transport_from_rate_converges_to_director_equation(oracle_mod):
    O = oracle_mod
    nx, ny, nz = 6, 5, 4
    base = dict(nx=nx, ny=ny, nz=nz, walls_z=False, K=0.03, q0=0.7, W0=0.01, gamma1=1.0, gamma2=-0.9,
                alpha1=0.1, alpha2=-0.95, alpha3=0.05, alpha4p=0.2, alpha5=0.45, alpha6=-0.45)
    n0 = I.random_director(nx, ny, nz, seed=11)
    u = I.random_velocity(nx, ny, nz, 1e-2, seed=12)
    diffs = []
    for dt in (4e-3, 2e-3, 1e-3):
        p = O.OracleParams(dt_fd=dt, n_from_rate=True, **base)
        n1, rate = O.fd_step(p, n0, u, return_rate=True)
        s_rate = O.stress(p, n1, u, rate)
        s_alg = O.stress(p, n1, u)
        assert np.max(np.abs(O.stress(p, n1, u, None) - s_alg)) == 0.0
        diffs.append(np.max(np.abs(s_rate - s_alg)) / np.max(np.abs(s_alg)))
    assert diffs[-1] < 1e-2
    for a, b in zip(diffs, diffs[1:]):
        assert 1.8 < a / b < 2.2  # first order in dt_FD


@pytest.mark.parametrize("ghost", ["zero", "mirror"])
def test_ghost_stress_total_force(oracle_mod, ghost):
    O = oracle_mod
    nx, ny, nz = 5, 4, 7
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=True, ghost_sigma=ghost)
    rng = np.random.default_rng(3)
    sig = rng.normal(size=(9, nx * ny * nz))
    F = O.force(p, sig)
    s3 = sig.reshape(3, 3, nz, ny * nx)
    factor = 1.0 if ghost == "mirror" else 0.5
    expect = factor * (np.sum(s3[:, 2, nz - 1], axis=-1) - np.sum(s3[:, 2, 0], axis=-1))
    assert np.max(np.abs(F.sum(axis=1) - expect)) < 1e-12
    uniform = np.repeat(rng.normal(size=(9, 1)), nx * ny * nz, axis=1)
    Fu = O.force(p, uniform)
    if ghost == "mirror":
        assert np.max(np.abs(Fu)) == 0.0
    else:
        assert np.max(np.abs(Fu)) > 0.1
