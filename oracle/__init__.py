"""FP64 CPU oracle for the hybrid LB + FD nematohydrodynamics step (arXiv:2503.06610).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_2503_06610_gb300`` and never imports it.

The per-site arithmetic lives in ``nh_oracle.c`` (plain C, double precision,
one site at a time, compiled without FMA contraction).  This module holds:

* ``build()`` - compile ``nh_oracle.c`` to ``oracle/_lib/liboracle.so``;
* thin ctypes wrappers of the C routines (arrays are numpy float64);
* ``OracleSim`` - the hybrid loop of Sec. II.D in the paper's order;
* diagnostics in numpy: mass, lattice Frank energy, tube centroids and the
  error metrics (relative L2 and the paper's epsilon of Sec. III.A).

Parity pins (see ``tests/test_oracle_*.py``) fix each routine against what the
paper and the mathematics determine; the coupled loop is held to the energy
dissipation and momentum balance of the Ericksen-Leslie equations, which fix
the sign and index placement of every coupling term, and to the linear theory
of a director wave coupled to shear flow, which fixes the size of the
backflow.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nh_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle in-tree (gcc, -O2, OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("walls_z", ctypes.c_int), ("anchoring", ctypes.c_int), ("shifted", ctypes.c_int),
        ("tau", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("K", ctypes.c_double), ("q0", ctypes.c_double),
        ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
        ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double), ("alpha3", ctypes.c_double),
        ("alpha4p", ctypes.c_double), ("alpha5", ctypes.c_double), ("alpha6", ctypes.c_double),
        ("W0", ctypes.c_double), ("dt_fd", ctypes.c_double),
        ("K11", ctypes.c_double), ("K22", ctypes.c_double), ("K33", ctypes.c_double),
        ("frank3", ctypes.c_int),
        ("solid", ctypes.c_void_p),
        ("renorm_predictor", ctypes.c_int), ("lap_wide", ctypes.c_int),
        ("n_from_rate", ctypes.c_int), ("ghost_sigma", ctypes.c_int),
    ]


@dataclass
class OracleParams:
    """Physical and lattice parameters, in lattice units (Delta x = Delta t = rho0 = 1)."""
    nx: int
    ny: int
    nz: int
    walls_z: bool = True
    anchoring: str = "homeotropic"  # "homeotropic" | "none"
    shifted: bool = True
    tau: float = 1.0
    g: tuple = (0.0, 0.0, 0.0)
    K: float = 0.0
    q0: float = 0.0
    gamma1: float = 1.0
    gamma2: float = 0.0
    alpha1: float = 0.0
    alpha2: float = 0.0
    alpha3: float = 0.0
    alpha4p: float = 0.0
    alpha5: float = 0.0
    alpha6: float = 0.0
    W0: float = 0.0
    dt_fd: int = 1
    paper_order: bool = False  # the loop order of Sec. II.D taken literally (see OracleSim)
    K11: float = None  # three-constant Frank energy when K11, K22, K33 are all given
    K22: float = None
    K33: float = None
    solid: object = None  # [N] uint8, 1 = solid node (obstacle); None: no obstacles
    # readings where the paper is silent (see nh_oracle.c)
    renorm_predictor: bool = False  # renormalise the predictor n^P too
    lap_wide: bool = False          # second derivatives as central differences of central differences
    n_from_rate: bool = False       # N of the stress from the corrector's averaged rate
    ghost_sigma: str = "zero"       # "zero" | "mirror": stress at the plates' ghost layers

    def __post_init__(self):
        if self.solid is not None:
            self.solid = np.ascontiguousarray(np.asarray(self.solid).reshape(-1), dtype=np.uint8)
            assert self.solid.size == self.N

    def fluid(self) -> np.ndarray:
        """[N] bool, True at fluid sites."""
        return np.ones(self.N, bool) if self.solid is None else self.solid == 0

    @property
    def frank3(self) -> bool:
        return self.K11 is not None and self.K22 is not None and self.K33 is not None

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def to_c(self) -> _Params:
        c = _Params()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        c.walls_z = 1 if self.walls_z else 0
        c.anchoring = 1 if self.anchoring == "homeotropic" else 0
        c.shifted = 1 if self.shifted else 0
        c.tau = self.tau
        c.g = (ctypes.c_double * 3)(*[float(v) for v in self.g])
        for k in ("K", "q0", "gamma1", "gamma2", "alpha1", "alpha2", "alpha3", "alpha4p",
                  "alpha5", "alpha6", "W0"):
            setattr(c, k, float(getattr(self, k)))
        c.dt_fd = float(self.dt_fd)
        if self.frank3:
            c.K11, c.K22, c.K33, c.frank3 = self.K11, self.K22, self.K33, 1
        if self.solid is not None:
            c.solid = self.solid.ctypes.data  # the array lives as long as these params
        c.renorm_predictor = 1 if self.renorm_predictor else 0
        c.lap_wide = 1 if self.lap_wide else 0
        c.n_from_rate = 1 if self.n_from_rate else 0
        c.ghost_sigma = {"zero": 0, "mirror": 1}[self.ghost_sigma] if isinstance(self.ghost_sigma, str) \
            else int(self.ghost_sigma)
        return c

    @classmethod
    def from_dict(cls, d: dict) -> "OracleParams":
        keys = {f for f in cls.__dataclass_fields__}
        return cls(**{k: v for k, v in d.items() if k in keys})


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        _lib.or_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(ctypes.c_int)]
        _lib.or_feq.argtypes = [ctypes.c_double, dp, ctypes.c_int, dp]
        _lib.or_guo_source.argtypes = [dp, dp, dp]
        _lib.or_lb_step.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        _lib.or_init_populations.argtypes = [pp, dp, dp, dp]
        _lib.or_molecular_field.argtypes = [pp, dp, dp]
        _lib.or_director_rate.argtypes = [pp, dp, dp, dp]
        _lib.or_fd_step.argtypes = [pp, dp, dp, dp]
        _lib.or_transport_point.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        _lib.or_viscous_stress_point.argtypes = [pp, dp, dp, dp, dp]
        _lib.or_elastic_stress_point.argtypes = [pp, dp, dp, dp]
        _lib.or_stress.argtypes = [pp, dp, dp, dp, dp]
        _lib.or_force.argtypes = [pp, dp, dp]
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_frank3_field.argtypes = [pp, dp, dp]
        _lib.or_frank3_field.restype = ctypes.c_double
        _lib.or_frank3_point.argtypes = [pp, dp, dp, dp, dp]
        _lib.or_frank3_point.restype = ctypes.c_double
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays are C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ lattice / point routines

def lattice():
    """(e[19,3] int, w[19], opp[19]) of the oracle's D3Q19 set."""
    e = (ctypes.c_int * 57)()
    w = np.zeros(19)
    opp = (ctypes.c_int * 19)()
    lib().or_lattice(e, _ptr(w), opp)
    return np.array(list(e), dtype=np.int64).reshape(19, 3), w, np.array(list(opp), dtype=np.int64)


def feq(rho: float, u, shifted: bool) -> np.ndarray:
    out = np.zeros(19)
    lib().or_feq(float(rho), _ptr(_f64(u)), 1 if shifted else 0, _ptr(out))
    return out


def guo_source(u, F) -> np.ndarray:
    out = np.zeros(19)
    lib().or_guo_source(_ptr(_f64(u)), _ptr(_f64(F)), _ptr(out))
    return out


def transport_point(n, h, D, gamma1, gamma2) -> np.ndarray:
    out = np.zeros(3)
    lib().or_transport_point(_ptr(_f64(n)), _ptr(_f64(h)), _ptr(_f64(np.ravel(D))), gamma1, gamma2, _ptr(out))
    return out


def viscous_stress_point(p: OracleParams, n, D, N) -> np.ndarray:
    out = np.zeros(9)
    c = p.to_c()
    lib().or_viscous_stress_point(ctypes.byref(c), _ptr(_f64(n)), _ptr(_f64(np.ravel(D))), _ptr(_f64(N)), _ptr(out))
    return out.reshape(3, 3)


def elastic_stress_point(p: OracleParams, n, dn) -> np.ndarray:
    """sigma^e for director n and gradient dn[b][g] = d_b n_g."""
    out = np.zeros(9)
    c = p.to_c()
    lib().or_elastic_stress_point(ctypes.byref(c), _ptr(_f64(n)), _ptr(_f64(np.ravel(dn))), _ptr(out))
    return out.reshape(3, 3)


# ------------------------------------------------------------------ field routines

def _vec(p: OracleParams, a) -> np.ndarray:
    a = _f64(a)
    assert a.size % p.N == 0
    return a


def init_populations(p: OracleParams, rho=None, u=None) -> np.ndarray:
    N = p.N
    rho = np.ones(N) if rho is None else _f64(np.ravel(rho))
    u = np.zeros(3 * N) if u is None else _f64(np.ravel(u))
    f = np.zeros(19 * N)
    c = p.to_c()
    lib().or_init_populations(ctypes.byref(c), _ptr(rho), _ptr(u), _ptr(f))
    return f.reshape(19, N)


def lb_step(p: OracleParams, f, Flc, Fu=None):
    """One LB step; returns (f_new[19,N], rho[N], u[3,N]).  Fu (optional) is
    the LC force whose half shifts u; by default the collision's force Flc."""
    N = p.N
    f = _f64(f)
    fnew = np.empty_like(f)
    rho = np.empty(N)
    u = np.empty(3 * N)
    c = p.to_c()
    fu = None if Fu is None else _vec(p, Fu)
    lib().or_lb_step(ctypes.byref(c), _ptr(f), _ptr(fnew), _ptr(_vec(p, Flc)),
                     _ptr(fu) if fu is not None else None, _ptr(rho), _ptr(u))
    return fnew.reshape(19, N), rho, u.reshape(3, N)


def molecular_field(p: OracleParams, n) -> np.ndarray:
    out = np.empty(3 * p.N)
    c = p.to_c()
    lib().or_molecular_field(ctypes.byref(c), _ptr(_vec(p, n)), _ptr(out))
    return out.reshape(3, p.N)


def director_rate(p: OracleParams, n, u) -> np.ndarray:
    out = np.empty(3 * p.N)
    c = p.to_c()
    lib().or_director_rate(ctypes.byref(c), _ptr(_vec(p, n)), _ptr(_vec(p, u)), _ptr(out))
    return out.reshape(3, p.N)


def fd_step(p: OracleParams, n, u, return_rate: bool = False):
    """One predictor-corrector FD step (Sec. II.B) + renormalisation; returns new n
    (and, with return_rate, the averaged time derivative that advanced it)."""
    n = _f64(n).copy()
    work = np.empty(9 * p.N)
    c = p.to_c()
    lib().or_fd_step(ctypes.byref(c), _ptr(n), _ptr(_vec(p, u)), _ptr(work))
    if return_rate:
        return n.reshape(3, p.N), work[:3 * p.N].reshape(3, p.N).copy()
    return n.reshape(3, p.N)


def stress(p: OracleParams, n, u, ndot=None) -> np.ndarray:
    """LC stress; ndot (the corrector's averaged rate) is used for N when p.n_from_rate."""
    out = np.empty(9 * p.N)
    c = p.to_c()
    nd = None if ndot is None else _vec(p, ndot)
    lib().or_stress(ctypes.byref(c), _ptr(_vec(p, n)), _ptr(_vec(p, u)), _ptr(nd) if nd is not None else None,
                    _ptr(out))
    return out.reshape(9, p.N)


def force(p: OracleParams, sigma) -> np.ndarray:
    out = np.empty(3 * p.N)
    c = p.to_c()
    lib().or_force(ctypes.byref(c), _ptr(_vec(p, sigma)), _ptr(out))
    return out.reshape(3, p.N)


def num_threads() -> int:
    return int(lib().or_num_threads())


# ------------------------------------------------------------------ hybrid loop (Sec. II.D)

@dataclass
class OracleSim:
    """The hybrid LB + FD loop of Sec. II.D, step by step.

    State: post-collision populations f (shifted or not), director n, the LC
    force F_lc frozen over each FD interval, and the latest moments rho, u.
    ``s`` counts completed LB steps.  After LB step s, if s % dt_fd == 0, the
    predictor-corrector runs with the u of that step, then the force is
    recomputed from the new n and that u.

    With ``paper_order`` the steps of Sec. II.D are taken in the printed order:
    streaming, macroscopic fields (u with the force in effect), the FD update
    and force when due, and only then the collision of that step, whose Guo
    source therefore carries the new force while its u still carries half of
    the old one.
    """
    p: OracleParams
    n: np.ndarray
    u: np.ndarray = None
    rho: np.ndarray = None
    f: np.ndarray = field(default=None, repr=False)
    F: np.ndarray = field(default=None, repr=False)
    s: int = 0
    ndot: np.ndarray = field(default=None, repr=False)  # averaged rate of the last FD update (n_from_rate)

    def __post_init__(self):
        N = self.p.N
        self.n = _f64(self.n).reshape(3, N).copy()
        self.u = np.zeros((3, N)) if self.u is None else _f64(self.u).reshape(3, N).copy()
        self.rho = np.ones(N) if self.rho is None else _f64(self.rho).reshape(N).copy()
        # Initialisation: populations at equilibrium, force from the initial fields.
        self.f = init_populations(self.p, self.rho, self.u)
        self.F = force(self.p, stress(self.p, self.n, self.u))

    def step(self, count: int = 1):
        for _ in range(count):
            due = (self.s + 1) % self.p.dt_fd == 0
            if self.p.paper_order and due:
                # macroscopic fields of this step (its collision result is not kept)
                _, self.rho, self.u = lb_step(self.p, self.f, self.F)
                self._fd_update()
                F_old = self.F
                self.F = force(self.p, stress(self.p, self.n, self.u, self.ndot))
                self.f, _, _ = lb_step(self.p, self.f, self.F, Fu=F_old)
                self.s += 1
                continue
            self.f, self.rho, self.u = lb_step(self.p, self.f, self.F)
            self.s += 1
            if due:
                self._fd_update()
                self.F = force(self.p, stress(self.p, self.n, self.u, self.ndot))
        return self

    def _fd_update(self):
        """Predictor-corrector on n with the current u; keeps the averaged rate for N (n_from_rate)."""
        self.n, rate = fd_step(self.p, self.n, self.u, return_rate=True)
        self.ndot = rate if self.p.n_from_rate else None

    def mass(self) -> float:
        return mass(self.p, self.f)

    def energy(self) -> float:
        return frank_energy(self.p, self.n)


# ------------------------------------------------------------------ diagnostics

def mass(p: OracleParams, f) -> float:
    """Total mass sum over fluid sites of sum_i f_i (the shifted store adds rho0 = 1 per site)."""
    fl = p.fluid()
    total = float(np.sum(np.asarray(f, dtype=np.float64).reshape(19, p.N)[:, fl]))
    return total + (float(fl.sum()) if p.shifted else 0.0)


def _ghosted(p: OracleParams, n) -> np.ndarray:
    """Director on (nz+2, ny, nx) with the z ghost layers of the wall reading."""
    n = np.asarray(n, dtype=np.float64).reshape(3, p.nz, p.ny, p.nx)
    if not p.walls_z:
        return np.concatenate([n[:, -1:], n, n[:, :1]], axis=1)
    if p.anchoring == "homeotropic":
        g = np.zeros((3, 1, p.ny, p.nx))
        g[2] = 1.0
        return np.concatenate([g, n, g], axis=1)
    return np.concatenate([n[:, :1], n, n[:, -1:]], axis=1)


def frank_energy(p: OracleParams, n) -> float:
    """Lattice Frank energy (Eq. free-energy-eq; one-constant form with K, plus
    the three-constant correction when K11, K22, K33 are given).

    E_d = sum over nearest-neighbour links (x, x+e_b) with at least one fluid
          end of  K/2 |n(x+e_b) - n(x)|^2 + K q0 eps_{a b c} n_a(x) n_c(x+e_b)
        + sum over fluid sites of  K q0^2 / 2 - (W0/2) n_z^2.
    Links to the wall ghost layers and to obstacle nodes (fixed directors) are
    included.  In a periodic box the chiral link sum equals sum_x n . curl_c n
    with the central curl, and -dE_d/dn is the molecular field h used by the
    director equation.
    """
    K, q0 = p.K, p.q0
    ng = _ghosted(p, n)                         # (3, nz+2, ny, nx)
    core = ng[:, 1:-1]
    solid = (~p.fluid()).reshape(p.nz, p.ny, p.nx)
    sg = np.concatenate([np.ones((1, p.ny, p.nx), bool), solid, np.ones((1, p.ny, p.nx), bool)], axis=0)
    E = 0.0
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0

    def links(lo, hi, keep, b):
        e = 0.5 * K * np.sum((hi - lo) ** 2, axis=0) + K * q0 * np.einsum("ac,a...,c...->...", eps[:, b, :], lo, hi)
        return float(np.sum(e[keep]))
    # x and y links (periodic)
    for b, axis in ((0, 3), (1, 2)):
        nb = np.roll(core, -1, axis=axis)
        E += links(core, nb, ~(solid & np.roll(solid, -1, axis=axis - 1)), b)
    # z links: (z, z+1) for z = -1 .. nz-1 with walls, z = 0 .. nz-1 periodic
    if p.walls_z:
        E += links(ng[:, :-1], ng[:, 1:], ~(sg[:-1] & sg[1:]), 2)
    else:
        E += links(core, np.roll(core, -1, axis=1), ~(solid & np.roll(solid, -1, axis=0)), 2)
    fl = p.fluid()
    nz_ = np.asarray(n, dtype=np.float64).reshape(3, -1)[2]
    E += float(fl.sum()) * 0.5 * K * q0 ** 2 - 0.5 * p.W0 * float(np.sum(nz_[fl] ** 2))
    if p.frank3:
        E += frank3_field(p, n)[0]
    return float(E)


def frank3_point(p: OracleParams, n3, G):
    """Delta f at one site for director n3[3] and gradient G[b][c] = d_b n_c:
    (Delta f, d Delta f/dn [3], d Delta f/dG [3][3])."""
    n3 = np.ascontiguousarray(n3, dtype=np.float64)
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(9))
    dfdn = np.empty(3)
    P = np.empty(9)
    c = p.to_c()
    f = lib().or_frank3_point(ctypes.byref(c), _ptr(n3), _ptr(G), _ptr(dfdn), _ptr(P))
    return float(f), dfdn, P.reshape(3, 3)


def frank3_field(p: OracleParams, n):
    """Three-constant correction: (sum over fluid sites of Delta f, its field
    -d(sum Delta f)/dn [3,N]).  Delta f = (K11-K)/2 (div n)^2 + (K22-K)/2
    (n . curl n + q0)^2 + (K33-K)/2 |n x curl n|^2 with central differences."""
    hd = np.empty(3 * p.N)
    c = p.to_c()
    E = lib().or_frank3_field(ctypes.byref(c), _ptr(_vec(p, n)), _ptr(hd))
    return float(E), hd.reshape(3, p.N)


def centroids(p: OracleParams, n, previous) -> np.ndarray:
    """Skyrmion-tube centroids by circular means of the weight w = (1 - n_z)/2.

    Each site is assigned to the nearest previous centroid (periodic distance);
    per tube, x_bar = Lx/(2 pi) * atan2(sum w sin(2 pi x/Lx), sum w cos(2 pi x/Lx)),
    likewise y_bar.  ``previous`` is a (T, 2) array; returns a (T, 2) array in [0, L).
    """
    n = np.asarray(n, dtype=np.float64).reshape(3, p.nz, p.ny, p.nx)
    w = 0.5 * (1.0 - n[2]) * p.fluid().reshape(p.nz, p.ny, p.nx)  # fluid sites only
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    prev = np.asarray(previous, dtype=np.float64).reshape(-1, 2)
    d2 = []
    for cx, cy in prev:
        dx = (x - cx + 0.5 * p.nx) % p.nx - 0.5 * p.nx
        dy = (y - cy + 0.5 * p.ny) % p.ny - 0.5 * p.ny
        d2.append(dx * dx + dy * dy)
    owner = np.argmin(np.stack(d2), axis=0)
    out = np.zeros_like(prev)
    for t in range(prev.shape[0]):
        m = owner == t
        ww = w[m]
        ax = 2 * np.pi * x[m] / p.nx
        ay = 2 * np.pi * y[m] / p.ny
        out[t, 0] = (np.arctan2(np.sum(ww * np.sin(ax)), np.sum(ww * np.cos(ax))) * p.nx / (2 * np.pi)) % p.nx
        out[t, 1] = (np.arctan2(np.sum(ww * np.sin(ay)), np.sum(ww * np.cos(ay))) * p.ny / (2 * np.pi)) % p.ny
    return out


def rel_l2(a, ref) -> float:
    """||a - ref||_2 / ||ref||_2 over all components."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))


def eps_paper(u, uref) -> float:
    """The paper's relative velocity error (Sec. III.A): sum_n |u - u_ref| / sum_n |u_ref|."""
    u = np.asarray(u, dtype=np.float64).reshape(3, -1)
    uref = np.asarray(uref, dtype=np.float64).reshape(3, -1)
    return float(np.sum(np.linalg.norm(u - uref, axis=0)) / np.sum(np.linalg.norm(uref, axis=0)))


def eps_component(u, uref, a: int) -> float:
    """Per-component form of epsilon (Sec. III.B)."""
    u = np.asarray(u, dtype=np.float64).reshape(3, -1)
    uref = np.asarray(uref, dtype=np.float64).reshape(3, -1)
    return float(np.sum(np.abs(u[a] - uref[a])) / np.sum(np.abs(uref[a])))
