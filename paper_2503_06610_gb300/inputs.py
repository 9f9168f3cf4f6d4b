"""Seeded synthetic inputs for the hybrid LB + FD nematohydrodynamics step.

This module only draws and lays out initial conditions and parameter sets; it
holds none of the method's arithmetic (no equilibrium, no molecular field, no
stress).  Both the CUDA library's callers and the FP64 CPU oracle take their
inputs from here, so the two start from identical bits.

Fields are numpy float64 arrays in structure-of-arrays layout ``[3][N]`` with
site index ``x + nx*(y + ny*z)``.

Workloads (the paper measures on no public dataset; everything is generated):

* tiny nematic channel 32x32x16: z_hat plus a 0.05 uniform random tilt;
* single skyrmion tube 96x96x32, q0 = 2 pi/32, radius 12, centred;
* multi-tube channel 256x256x64, q0 = 2 pi/64, 8 tubes of radius 20 at seeded
  non-overlapping centres;
* batched sweep: 64 channels with lateral L in {32,48,64,96}, Lz in {16,24,32},
  g_x log-uniform in [1e-7, 1e-5], pitch p uniform in [Lz, 2 Lz], one tube each.
"""
from __future__ import annotations

import math

import numpy as np

# Leslie viscosities for a flow-alignment parameter gamma2/gamma1 = -0.9 with
# gamma1 = 1: alpha3 - alpha2 = gamma1, alpha3 + alpha2 = gamma2 (Sec. II.A),
# Parodi alpha6 - alpha5 = gamma2; alpha1 = alpha4' = 0.
LESLIE_ALIGN_09 = dict(gamma1=1.0, gamma2=-0.9, alpha1=0.0, alpha2=-0.95, alpha3=0.05,
                       alpha4p=0.0, alpha5=0.45, alpha6=-0.45)


# gamma2/gamma1 = -0.5 with gamma1 = 1 and alpha5 = -alpha6 = 1/4 (Parodi holds):
# with the LB viscosity of tau = 1 (alpha4 = 2 (tau - 1/2)/3 = 1/3) these satisfy
# Leslie's inequalities, so the Ericksen-Leslie dissipation is positive
# definite (gamma1 (2 alpha4 + alpha5 + alpha6) = 2/3 > gamma2^2 = 1/4).
LESLIE_DISSIPATIVE = dict(gamma1=1.0, gamma2=-0.5, alpha1=0.0, alpha2=-0.75, alpha3=0.25,
                          alpha4p=0.0, alpha5=0.25, alpha6=-0.25)


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def _pack(nx_, ny_, nz_):
    return np.stack([nx_.ravel(), ny_.ravel(), nz_.ravel()]).astype(np.float64)


def uniform_director(nx, ny, nz, direction=(0.0, 0.0, 1.0)):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    N = nx * ny * nz
    return np.repeat(d[:, None], N, axis=1)


def tilted_director(nx, ny, nz, amplitude=0.05, seed=0):
    """n = normalise(a xi_x, a xi_y, 1), xi ~ U(-1, 1) from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = nx * ny * nz
    xi = rng.uniform(-1.0, 1.0, size=(2, N))
    n = np.stack([amplitude * xi[0], amplitude * xi[1], np.ones(N)])
    return n / np.linalg.norm(n, axis=0, keepdims=True)


def distorted_director(nx, ny, nz, tilt=0.6, swing=0.4, twist=0.5):
    """Smooth splay-bend-twist field: polar angle tilt sin(2 pi x/nx) + swing cos(2 pi y/ny),
    azimuth twist sin(2 pi z/nz + 0.3); one period per axis, so periodic in x, y and z."""
    x, y, z = _grid(nx, ny, nz)
    a = tilt * np.sin(2 * math.pi * x / nx) + swing * np.cos(2 * math.pi * y / ny)
    b = twist * np.sin(2 * math.pi * z / nz + 0.3)
    return _pack(np.sin(a) * np.cos(b), np.sin(a) * np.sin(b), np.cos(a))


def skyrmion_tubes(nx, ny, nz, centres, radius, handedness=1.0):
    """Extruded 2D skyrmion ansatz: radial pi-twist of radius R around each centre.

    n = (-s sin(theta) sin(phi), s sin(theta) cos(phi), cos(theta)),
    theta(r) = pi (1 - r/R) for r < R, else 0, with r and phi about the nearest
    centre (periodic minimum image in x and y) and s = handedness = +-1.
    """
    x, y, _ = _grid(nx, ny, nz)
    best_r = np.full(x.shape, np.inf)
    best_dx = np.zeros_like(x)
    best_dy = np.zeros_like(x)
    for cx, cy in centres:
        dx = (x - cx + 0.5 * nx) % nx - 0.5 * nx
        dy = (y - cy + 0.5 * ny) % ny - 0.5 * ny
        r = np.hypot(dx, dy)
        m = r < best_r
        best_r = np.where(m, r, best_r)
        best_dx = np.where(m, dx, best_dx)
        best_dy = np.where(m, dy, best_dy)
    theta = np.where(best_r < radius, math.pi * (1.0 - best_r / radius), 0.0)
    phi = np.arctan2(best_dy, best_dx)
    s = float(handedness)
    return _pack(-s * np.sin(theta) * np.sin(phi), s * np.sin(theta) * np.cos(phi), np.cos(theta))


def place_tubes(nx, ny, count, radius, seed=0, max_tries=100000):
    """Seeded rejection sampling of tube centres with periodic distance >= 2R."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place non-overlapping tubes")
        c = (float(rng.uniform(0, nx)), float(rng.uniform(0, ny)))
        ok = True
        for (px, py) in centres:
            dx = (c[0] - px + 0.5 * nx) % nx - 0.5 * nx
            dy = (c[1] - py + 0.5 * ny) % ny - 0.5 * ny
            if dx * dx + dy * dy < (2 * radius) ** 2:
                ok = False
                break
        if ok:
            centres.append(c)
    return centres


def twist_mode(nx, ny, nz, amplitude=1e-3, wavenumber=None):
    """n = (0, cos theta, sin theta), theta = a sin(k x), k = 2 pi / nx by default."""
    k = 2 * math.pi / nx if wavenumber is None else wavenumber
    x, _, _ = _grid(nx, ny, nz)
    th = amplitude * np.sin(k * x)
    return _pack(np.zeros_like(th), np.cos(th), np.sin(th))


def helix(nx, ny, nz, q):
    """Cholesteric helix along z: n = (cos q z, sin q z, 0)."""
    _, _, z = _grid(nx, ny, nz)
    return _pack(np.cos(q * z), np.sin(q * z), np.zeros_like(z))


def shear_wave(nx, ny, nz, amplitude, wavenumber=None):
    """u = (U sin(k z), 0, 0), k = 2 pi / nz by default (periodic box)."""
    k = 2 * math.pi / nz if wavenumber is None else wavenumber
    _, _, z = _grid(nx, ny, nz)
    ux = amplitude * np.sin(k * z)
    return _pack(ux, np.zeros_like(ux), np.zeros_like(ux))


def random_director(nx, ny, nz, seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=(3, nx * ny * nz))
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def random_velocity(nx, ny, nz, amplitude, seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return amplitude * rng.uniform(-1.0, 1.0, size=(3, nx * ny * nz))


# ------------------------------------------------------------------ workload presets

def tiny_channel(shifted=True):
    """32x32x16 nematic channel, tau=1, g_x=1e-6, K=0.04, gamma2/gamma1=-0.9, q0=0."""
    params = dict(nx=32, ny=32, nz=16, walls_z=True, anchoring="homeotropic", shifted=shifted,
                  tau=1.0, g=(1e-6, 0.0, 0.0), K=0.04, q0=0.0, W0=0.0, dt_fd=1, **LESLIE_ALIGN_09)
    n0 = tilted_director(32, 32, 16, amplitude=0.05, seed=0)
    return params, n0


def skyrmion_channel(gx=1e-5, dt_fd=1, shifted=True, K=0.005, nx=96, ny=96, nz=32, radius=12.0):
    """Single skyrmion tube in Poiseuille flow, 96x96x32, q0 = 2 pi/32."""
    params = dict(nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="homeotropic", shifted=shifted,
                  tau=1.0, g=(gx, 0.0, 0.0), K=K, q0=2 * math.pi / 32, W0=0.0, dt_fd=dt_fd,
                  **LESLIE_ALIGN_09)
    n0 = skyrmion_tubes(nx, ny, nz, [(nx / 2, ny / 2)], radius)
    return params, n0


def multi_tube_channel(dt_fd=16, shifted=True, K=0.005, seed=0, nx=256, ny=256, nz=64, tubes=8,
                       radius=20.0, gx=1e-5):
    """256x256x64, q0 = 2 pi/64, 8 tubes of radius 20 at seeded centres."""
    params = dict(nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="homeotropic", shifted=shifted,
                  tau=1.0, g=(gx, 0.0, 0.0), K=K, q0=2 * math.pi / 64, W0=0.0, dt_fd=dt_fd,
                  **LESLIE_ALIGN_09)
    centres = place_tubes(nx, ny, tubes, radius, seed=seed)
    n0 = skyrmion_tubes(nx, ny, nz, centres, radius)
    return params, n0, centres


def batched_sweep(count=64, seed=0, K=0.005, dt_fd=16):
    """64 channels of uneven size with one tube each; returns a list of (params, n0, centre)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        L = int(rng.choice([32, 48, 64, 96]))
        Lz = int(rng.choice([16, 24, 32]))
        gx = float(10 ** rng.uniform(-7, -5))
        pitch = float(rng.uniform(Lz, 2 * Lz))
        R = 0.25 * L
        params = dict(nx=L, ny=L, nz=Lz, walls_z=True, anchoring="homeotropic", shifted=True,
                      tau=1.0, g=(gx, 0.0, 0.0), K=K, q0=2 * math.pi / pitch, W0=0.0, dt_fd=dt_fd,
                      **LESLIE_ALIGN_09)
        n0 = skyrmion_tubes(L, L, Lz, [(L / 2, L / 2)], R)
        out.append((params, n0, (L / 2, L / 2)))
    return out


# ------------------------------------------------------------------ warm-start network inputs

# Layer widths of the warm-start U-Net (name, cin, cout) in parameter order; the
# head is a 1x1x1 convolution 16 -> 3.  Weights are W[tap][cout][cin] then bias.
UNET_CONV_LAYERS = [
    ("enc1a", 16, 16), ("enc1b", 16, 16), ("enc2a", 16, 16), ("enc2b", 16, 16),
    ("enc3a", 16, 32), ("enc3b", 32, 32), ("bota", 32, 64), ("botb", 64, 64),
    ("dec3a", 96, 32), ("dec3b", 32, 32), ("dec2a", 48, 16), ("dec2b", 16, 16),
    ("dec1a", 32, 16), ("dec1b", 16, 16),
]
UNET_HEAD = (16, 3)


def unet_init_params(seed=0):
    """He-normal conv weights (std sqrt(2 / (27 cin))), zero biases, a small head (std 1e-2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, ci, co in UNET_CONV_LAYERS:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), size=27 * co * ci))
        parts.append(np.zeros(co))
    ci, co = UNET_HEAD
    parts.append(rng.normal(0.0, 1e-2, size=ci * co))
    parts.append(np.zeros(co))
    return np.concatenate(parts)


def warmstart_samples(count, seed=0, nx=64, ny=64, lz_choices=(32,), K=0.005, dt_fd=30):
    """Seeded relaxation problems for the learned warm start, in the paper's
    skyrmion setup (Sec. III.A): no anchoring at the plates and a weak bulk
    anchoring W0 along z.  Per sample: cell thickness Lz, pitch P ~ U[20, 40]
    (q0 = 2 pi / P), W0 = w K q0^2 with w ~ U[3, 3.8] (the uniform background is
    then the ground state, kappa = pi^2 K q0^2 / (4 W0) < 1, and an isolated tube
    is metastable; for w < pi^2/4 the ground state is helical and tubes unwind,
    and for w above about 4 the relaxed tube is a few sites wide and collapses
    on the lattice), tube radius R ~ U[0.3, 0.5] P; one tube centred on the
    site (nx/2, ny/2), fluid at rest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        lz = int(rng.choice(lz_choices))
        pitch = float(rng.uniform(20.0, 40.0))
        q0 = 2 * math.pi / pitch
        w0 = float(rng.uniform(3.0, 3.8) * K * q0 * q0)
        radius = float(pitch * rng.uniform(0.3, 0.5))
        params = dict(nx=nx, ny=ny, nz=lz, walls_z=True, anchoring="none", shifted=True, tau=1.0,
                      g=(0.0, 0.0, 0.0), K=K, q0=q0, W0=w0, dt_fd=dt_fd, **LESLIE_ALIGN_09)
        n0 = skyrmion_tubes(nx, ny, lz, [(nx // 2, ny // 2)], radius)
        out.append((params, n0))
    return out


# ------------------------------------------------------------------ paper regime (Table I)

def table1_regime(nx=64, ny=64, nz=16, dt_fd=250, split=0.3, lb_share=None, radius=7.0, shifted=True,
                  paper_order=True):
    """The paper's test case in lattice units: Table I (MBBA, doubled alpha4),
    pitch P = 14, 64x64x16 (Sec. III.A), g = 2e-9, no anchoring at the plates
    with bulk W0 = 1.5e-8.  The one-constant K is the mean of K11, K22, K33;
    gamma1 = alpha3 - alpha2, gamma2 = alpha3 + alpha2.  The isotropic viscosity
    alpha4 is shared between the FD force (alpha4' = split * alpha4) and the
    lattice Boltzmann fluid (2 rho c_s^2 (tau - 1/2) = (1 - split) alpha4, which
    fixes tau; lb_share overrides that share).  Sec. II.B asks that the two
    parts add up to alpha4 and that they be equal.  The FD force is explicit
    and held for dt_FD LB steps, and over a long interval its viscous part
    hands a velocity mode back with the ratio alpha4' / (2 rho c_s^2 (tau -
    1/2)) of the two viscosities and the opposite sign: equal shares (split =
    0.5) are marginal and leave the tube state for dt_FD >= 10.  split = 0.3
    (tau = 1.478) runs the whole dt_FD range of Sec. III.B, 1 to 5000; 0.15
    fails at dt_FD = 1 instead.

    paper_order = True runs the loop of Sec. II.D in its printed order: the
    FD update and the force come between the macroscopic fields and the
    collision of the same step.  With the fused order (the collision keeps the
    force of the previous interval) the force lags the velocity it is computed
    from by one LB step, and at odd dt_FD that lag feeds a lattice mode of
    wavevector (pi/2, pi/2, pi/2) that flips sign every step, through the
    central differences of the viscous stress; with these viscosities it grows
    until the run diverges.  Even dt_FD samples that mode in phase and does
    not feed it.

    The tube is the radial pi-twist ansatz of radius P/2 (the cited ansatz is
    not available)."""
    K11, K22, K33 = 1.67e-7, 7.88e-8, 2.62e-7
    a1, a2, a3, a4, a5, a6 = 0.0373, -0.4496, -0.0203, 0.9318, 0.3084, -0.1617
    tau = 0.5 + 1.5 * ((1.0 - split) if lb_share is None else lb_share) * a4
    params = dict(nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="none", shifted=shifted, tau=tau,
                  g=(2e-9, 0.0, 0.0), K=(K11 + K22 + K33) / 3.0, q0=2 * math.pi / 14.0, W0=1.5e-8,
                  dt_fd=dt_fd, gamma1=a3 - a2, gamma2=a3 + a2, alpha1=a1, alpha2=a2, alpha3=a3,
                  alpha4p=split * a4, alpha5=a5, alpha6=a6, paper_order=paper_order)
    n0 = skyrmion_tubes(nx, ny, nz, [(nx / 2, ny / 2)], radius)
    return params, n0
