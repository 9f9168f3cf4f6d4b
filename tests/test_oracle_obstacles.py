"""Pins of the oracle's obstacles (solid nodes with bounce-back and fixed,
infinitely anchored directors; arXiv:2503.06610, Sec. II.B).

* A channel whose plates are two layers of solid nodes normal to y, in a box
  periodic in every direction, is the z-plate channel (already pinned against
  Poiseuille, mass conservation and the energy gradient) seen in rotated axes:
  after the cyclic permutation (x, y, z) -> (Z, X, Y) of sites and vector
  components, the two runs agree to rounding in n, u and rho, in mass and in
  energy.
* Mass over the fluid sites is conserved around an obstacle under a body force.
* h = -dE_d/dn at the fluid sites with a random obstacle (brute force).
"""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

LESLIE = I.LESLIE_ALIGN_09


def _to_B(a, nxA, nyA, nzA, vector):
    """A field on A's sites (x, y, z) -> B's sites (X, Y, Z) = (y, z + 1, x) of
    a (nyA) x (nzA + 2) x (nxA) box; vector components (v_y, v_z, v_x)."""
    if vector:
        a = np.asarray(a).reshape(3, nzA, nyA, nxA)
        comps = [a[1], a[2], a[0]]
        return np.stack([_to_B(c, nxA, nyA, nzA, False) for c in comps])
    a = np.asarray(a).reshape(nzA, nyA, nxA)       # [z][y][x]
    out = np.zeros((nxA, nzA + 2, nyA))            # B layout [Z][Y][X]
    out[:, 1:-1, :] = np.transpose(a, (2, 0, 1))   # Z = x, Y = z + 1, X = y
    return out


def test_solid_plates_equal_rotated_walls(oracle_mod):
    O = oracle_mod
    nxA, nyA, nzA = 8, 6, 5
    dA = dict(nx=nxA, ny=nyA, nz=nzA, walls_z=True, anchoring="homeotropic", shifted=True, tau=0.8,
              g=(2e-5, -1e-5, 3e-6), K=0.03, q0=2 * math.pi / 9, W0=0.0, dt_fd=2, **dict(LESLIE, alpha4p=0.02))
    # (W0 = 0: the bulk anchoring W0 n_z z_hat singles out z and does not rotate with the box)
    n0A = I.skyrmion_tubes(nxA, nyA, nzA, [(4.0, 3.0)], 2.5)
    u0A = I.random_velocity(nxA, nyA, nzA, 1e-3, seed=2)
    # B: periodic box, solid layers at Y = 0 and Y = nzA + 1 holding n = e_Y (A's z_hat)
    solid = np.zeros((nxA, nzA + 2, nyA), np.uint8)
    solid[:, 0, :] = 1
    solid[:, -1, :] = 1
    n0B = _to_B(n0A, nxA, nyA, nzA, True)
    n0B[1][solid == 1] = 1.0
    u0B = _to_B(u0A, nxA, nyA, nzA, True)
    dB = dict(dA, nx=nyA, ny=nzA + 2, nz=nxA, walls_z=False, g=(dA["g"][1], dA["g"][2], dA["g"][0]))
    pA = O.OracleParams(**dA)
    pB = O.OracleParams(solid=solid, **dB)
    a = O.OracleSim(pA, n0A, u=u0A).step(9)
    b = O.OracleSim(pB, n0B.reshape(3, -1), u=u0B.reshape(3, -1)).step(9)
    fl = solid.reshape(-1) == 0
    for fa, fb, vec in ((a.n, b.n, True), (a.u, b.u, True), (a.rho, b.rho, False)):
        ref = _to_B(fa, nxA, nyA, nzA, vec).reshape(3 if vec else 1, -1)[:, fl]
        got = np.asarray(fb).reshape(3 if vec else 1, -1)[:, fl]
        assert np.max(np.abs(got - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))
    assert np.array_equal(b.n[:, ~fl], n0B.reshape(3, -1)[:, ~fl])       # fixed directors
    assert np.max(np.abs(b.u[:, ~fl])) == 0.0
    assert abs(a.mass() - b.mass()) < 1e-12 * pA.N
    assert abs(O.frank_energy(pA, a.n) - O.frank_energy(pB, b.n)) < 1e-12 * abs(O.frank_energy(pA, a.n))


def _sphere(nx, ny, nz, c, r):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) <= r * r).astype(np.uint8)


def _normals(solid, c):
    nz, ny, nx = solid.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = np.stack([x - c[0], y - c[1], z - c[2]]).astype(float)
    v[:, np.linalg.norm(v, axis=0) == 0] = np.array([0, 0, 1.0])[:, None]
    return v / np.linalg.norm(v, axis=0)


def test_mass_conserved_around_obstacle(oracle_mod):
    O = oracle_mod
    nx, ny, nz = 12, 10, 8
    solid = _sphere(nx, ny, nz, (6, 5, 4), 2.5)
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=True, shifted=True, tau=0.7, g=(1e-4, 2e-5, 0.0),
                       K=0.02, q0=0.3, dt_fd=3, solid=solid, **LESLIE)
    n0 = I.tilted_director(nx, ny, nz, amplitude=0.3, seed=1).reshape(3, nz, ny, nx)
    n0[:, solid == 1] = _normals(solid, (6, 5, 4))[:, solid == 1]
    sim = O.OracleSim(p, n0.reshape(3, -1))
    m0 = sim.mass()
    sim.step(40)
    assert abs(sim.mass() - m0) < 1e-12 * p.N
    fl = solid.reshape(-1) == 0
    assert np.max(np.abs(sim.u[:, ~fl])) == 0.0
    assert np.max(np.abs(sim.u[:, fl])) > 1e-4


def test_field_is_energy_gradient_with_obstacle(oracle_mod):
    O = oracle_mod
    nx, ny, nz = 5, 4, 4
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[1:3, 1:3, 2] = 1
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="homeotropic", K=0.7, q0=0.9, W0=0.3,
                       solid=solid)
    n = I.random_director(nx, ny, nz, seed=4)
    h = O.molecular_field(p, n)
    fl = solid.reshape(-1) == 0
    d = 1e-6
    for a in range(3):
        for s in np.flatnonzero(fl):
            npl = n.copy()
            npl[a, s] += d
            nm = n.copy()
            nm[a, s] -= d
            g = (O.frank_energy(p, npl) - O.frank_energy(p, nm)) / (2 * d)
            assert abs(g + h[a, s]) < 1e-7 * np.max(np.abs(h))
