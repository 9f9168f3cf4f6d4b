"""Python binding of the C ABI in ``include/nh.h`` (ctypes; argument marshalling only).

Every computation runs in the CUDA library ``_lib/libnh.so``; this module only
converts arguments.  PyTorch provides device memory (the context workspace)
and streams.  There is no CPU fallback: if the library or a GPU is missing the
calls raise.

Low-level functions carry the C names (``nh_create``, ``nh_set_fields``,
``nh_step``, ``nh_batch_step``, ``nh_get_fields``, ``nh_diagnostics``,
``nh_destroy`` ...).  ``Channel`` wraps one context together with its torch
workspace for convenience.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

NH_OK = 0
NH_EINVAL = -1
NH_ECUDA = -2
NH_ENOMEM = -3
NH_EUNSTABLE = -4
NH_ETIMEOUT = -5

NH_FP64, NH_FP32 = 0, 1
NH_STORE_F64, NH_STORE_F32, NH_STORE_F16S, NH_STORE_BF16S = 0, 1, 2, 3
NH_ANCHOR_NONE, NH_ANCHOR_HOMEOTROPIC = 0, 1
NH_MAX_TUBES = 32
KCLASSES = ("lb", "fd_predict", "fd_correct", "stress", "force")

STORAGE = {"f64": NH_STORE_F64, "f32": NH_STORE_F32, "f16s": NH_STORE_F16S, "bf16s": NH_STORE_BF16S}
PRECISION = {"fp64": NH_FP64, "fp32": NH_FP32}


class NHError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class nh_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("walls_z", ctypes.c_int32), ("anchoring", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("storage", ctypes.c_int32), ("shifted", ctypes.c_int32),
        ("dt_fd", ctypes.c_int32), ("check_stability", ctypes.c_int32),
        ("paper_order", ctypes.c_int32), ("frank3", ctypes.c_int32),
        ("renorm_predictor", ctypes.c_int32), ("lap_wide", ctypes.c_int32),
        ("n_from_rate", ctypes.c_int32), ("ghost_sigma", ctypes.c_int32),
        ("tau", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("K", ctypes.c_double), ("q0", ctypes.c_double),
        ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
        ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double), ("alpha3", ctypes.c_double),
        ("alpha4p", ctypes.c_double), ("alpha5", ctypes.c_double), ("alpha6", ctypes.c_double),
        ("W0", ctypes.c_double),
        ("K11", ctypes.c_double), ("K22", ctypes.c_double), ("K33", ctypes.c_double),
    ]


class nh_diag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("mass", ctypes.c_double), ("energy", ctypes.c_double),
        ("max_u", ctypes.c_double), ("min_norm", ctypes.c_double), ("max_norm", ctypes.c_double),
        ("nonfinite", ctypes.c_int32), ("n_tubes", ctypes.c_int32),
        ("centroid", (ctypes.c_double * 2) * NH_MAX_TUBES),
        ("tube_weight", ctypes.c_double * NH_MAX_TUBES),
    ]


class nh_row_copy(ctypes.Structure):
    _fields_ = [("src_slab", ctypes.c_int32), ("src_row", ctypes.c_int32),
                ("dst_slab", ctypes.c_int32), ("dst_row", ctypes.c_int32), ("comp_mask", ctypes.c_uint32)]


NH_HALO_POPULATIONS, NH_HALO_VECTOR, NH_HALO_STRESS = 0, 1, 2


class nh_timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 5), ("ms", ctypes.c_double * 5)]


# Every symbol of include/nh.h with its signature.
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "nh_error_string": ([ctypes.c_int], ctypes.c_char_p),
    "nh_last_error": ([_VP], ctypes.c_char_p),
    "nh_workspace_bytes": ([ctypes.POINTER(nh_params), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "nh_create": ([ctypes.POINTER(nh_params), _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "nh_bind_workspace": ([_VP, _VP, ctypes.c_size_t], ctypes.c_int),
    "nh_set_fields": ([_VP, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "nh_get_fields": ([_VP, _VP, _VP, _VP, ctypes.c_int], ctypes.c_int),
    "nh_get_populations": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "nh_set_populations": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "nh_get_force": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "nh_restore": ([_VP, _VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
    "nh_step": ([_VP, ctypes.c_int64, _VP], ctypes.c_int),
    "nh_fd_update": ([_VP, _VP], ctypes.c_int),
    "nh_batch_step": ([ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int64, _VP], ctypes.c_int),
    "nh_batch_autotune": ([ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "nh_set_tubes": ([_VP, _DP, ctypes.c_int], ctypes.c_int),
    "nh_set_solid": ([_VP, _VP, ctypes.c_int], ctypes.c_int),
    "nh_relax": ([_VP, ctypes.c_int64, _VP], ctypes.c_int),
    "nh_director_change": ([_VP, _DP], ctypes.c_int),
    "nh_symmetrize_c4": ([_VP], ctypes.c_int),
    "nh_batch_relax": ([ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int64, _VP], ctypes.c_int),
    "nh_diagnostics": ([_VP, ctypes.POINTER(nh_diag)], ctypes.c_int),
    "nh_diagnostics_enqueue": ([_VP, _VP], ctypes.c_int),
    "nh_diagnostics_read": ([_VP, ctypes.POINTER(nh_diag)], ctypes.c_int),
    "nh_set_timing": ([_VP, ctypes.c_int], ctypes.c_int),
    "nh_get_timing": ([_VP, ctypes.POINTER(nh_timing)], ctypes.c_int),
    "nh_launch_count": ([_VP], ctypes.c_int64),
    "nh_set_graphs": ([_VP, ctypes.c_int], ctypes.c_int),
    "nh_set_wait_limit": ([_VP, ctypes.c_double], ctypes.c_int),
    "nh_set_diag_fold": ([_VP, ctypes.c_int], ctypes.c_int),
    "nh_set_lb_variant": ([_VP, ctypes.c_int], ctypes.c_int),
    "nh_set_fd_variant": ([_VP, ctypes.c_int], ctypes.c_int),
    "nh_autotune": ([_VP, _VP, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "nh_destroy": ([_VP], None),
    "nh_unet_param_count": ([], ctypes.c_int64),
    "nh_unet_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)], ctypes.c_int),
    "nh_unet_workspace_bytes": ([_VP, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "nh_unet_bind": ([_VP, _VP, ctypes.c_size_t], ctypes.c_int),
    "nh_unet_set_params": ([_VP, _VP, _VP], ctypes.c_int),
    "nh_unet_forward": ([_VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "nh_unet_backward": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "nh_unet_activation": ([_VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "nh_unet_adam": ([_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int, ctypes.c_float, _VP], ctypes.c_int),
    "nh_unet_destroy": ([_VP], None),
    "nh_unet_status": ([_VP, _VP], ctypes.c_int),
    "nh_diagnostics_noalloc": ([ctypes.POINTER(nh_params), _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "nh_slab_plan": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.POINTER(nh_row_copy),
                      ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "nh_slab_init": ([ctypes.POINTER(_VP), ctypes.c_int, _VP], ctypes.c_int),
    "nh_slab_step": ([ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int64, _VP], ctypes.c_int),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``libnh.so`` (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run the package build)")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(code, ctx=None):
    if code != NH_OK:
        lib = load_library()
        msg = lib.nh_last_error(ctx)
        raise NHError(code, (msg or b"").decode() or lib.nh_error_string(code).decode())
    return code


def make_params(d: dict) -> nh_params:
    """nh_params from a dict with the oracle's keys plus precision / storage."""
    p = nh_params()
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
    p.walls_z = 1 if d.get("walls_z", True) else 0
    anch = d.get("anchoring", "homeotropic")
    p.anchoring = NH_ANCHOR_HOMEOTROPIC if anch in ("homeotropic", NH_ANCHOR_HOMEOTROPIC) else NH_ANCHOR_NONE
    prec = d.get("precision", "fp32")
    p.precision = PRECISION[prec] if isinstance(prec, str) else int(prec)
    default_store = "f64" if p.precision == NH_FP64 else "f32"
    st = d.get("storage", default_store)
    p.storage = STORAGE[st] if isinstance(st, str) else int(st)
    p.shifted = 1 if d.get("shifted", True) else 0
    p.dt_fd = int(d.get("dt_fd", 1))
    p.check_stability = 1 if d.get("check_stability", False) else 0
    p.paper_order = 1 if d.get("paper_order", False) else 0
    for k in ("renorm_predictor", "lap_wide", "n_from_rate"):
        v = d.get(k, False)
        setattr(p, k, int(v) if not isinstance(v, bool) else (1 if v else 0))
    gs = d.get("ghost_sigma", "zero")
    p.ghost_sigma = {"zero": 0, "mirror": 1}[gs] if isinstance(gs, str) else int(gs)
    if d.get("K11") is not None and d.get("K22") is not None and d.get("K33") is not None:
        p.frank3 = 1
        p.K11, p.K22, p.K33 = float(d["K11"]), float(d["K22"]), float(d["K33"])
    p.tau = float(d.get("tau", 1.0))
    g = d.get("g", (0.0, 0.0, 0.0))
    p.g = (ctypes.c_double * 3)(*[float(v) for v in g])
    for k, default in (("K", 0.0), ("q0", 0.0), ("gamma1", 1.0), ("gamma2", 0.0), ("alpha1", 0.0),
                       ("alpha2", 0.0), ("alpha3", 0.0), ("alpha4p", 0.0), ("alpha5", 0.0),
                       ("alpha6", 0.0), ("W0", 0.0)):
        setattr(p, k, float(d.get(k, default)))
    return p


# ------------------------------------------------------------------ thin C-name wrappers

def nh_workspace_bytes(p: nh_params) -> int:
    lib = load_library()
    out = ctypes.c_size_t(0)
    _check(lib.nh_workspace_bytes(ctypes.byref(p), ctypes.byref(out)))
    return int(out.value)


def nh_create(p: nh_params, stream=None):
    lib = load_library()
    h = _VP()
    _check(lib.nh_create(ctypes.byref(p), _VP(stream or 0), ctypes.byref(h)))
    return h


def nh_bind_workspace(ctx, ptr: int, nbytes: int):
    _check(load_library().nh_bind_workspace(ctx, _VP(ptr), nbytes), ctx)


def _ptr_of(a, on_device):
    if a is None:
        return None
    if on_device:
        return _VP(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return _VP(a.ctypes.data)


def nh_set_fields(ctx, n, u=None, rho=None, on_device=False):
    _check(load_library().nh_set_fields(ctx, _ptr_of(n, on_device), _ptr_of(u, on_device),
                                        _ptr_of(rho, on_device), 1 if on_device else 0), ctx)


def nh_get_fields(ctx, n=None, u=None, rho=None, on_device=False):
    _check(load_library().nh_get_fields(ctx, _ptr_of(n, on_device), _ptr_of(u, on_device),
                                        _ptr_of(rho, on_device), 1 if on_device else 0), ctx)


def nh_get_populations(ctx, f, on_device=False):
    _check(load_library().nh_get_populations(ctx, _ptr_of(f, on_device), 1 if on_device else 0), ctx)


def nh_set_populations(ctx, f, on_device=False):
    _check(load_library().nh_set_populations(ctx, _ptr_of(f, on_device), 1 if on_device else 0), ctx)


def nh_get_force(ctx, F, on_device=False):
    _check(load_library().nh_get_force(ctx, _ptr_of(F, on_device), 1 if on_device else 0), ctx)


def nh_restore(ctx, n, F=None, u=None, rho=None, step=0, on_device=False):
    _check(load_library().nh_restore(ctx, _ptr_of(n, on_device), _ptr_of(F, on_device), _ptr_of(u, on_device),
                                     _ptr_of(rho, on_device), int(step), 1 if on_device else 0), ctx)


def nh_step(ctx, n_lb_steps: int, stream=None):
    _check(load_library().nh_step(ctx, int(n_lb_steps), _VP(stream or 0)), ctx)


def nh_fd_update(ctx, stream=None):
    _check(load_library().nh_fd_update(ctx, _VP(stream or 0)), ctx)


def nh_batch_step(ctxs, n_lb_steps: int, stream=None):
    arr = (_VP * len(ctxs))(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    _check(load_library().nh_batch_step(arr, len(ctxs), int(n_lb_steps), _VP(stream or 0)))


def nh_slab_plan(ny_local, kind):
    """Halo plan of slabs with ny_local interior rows each: a list of
    (src_slab, src_row, dst_slab, dst_row, [components])."""
    lib = load_library()
    arr = (ctypes.c_int32 * len(ny_local))(*[int(v) for v in ny_local])
    n = ctypes.c_int(0)
    _check(lib.nh_slab_plan(len(ny_local), arr, int(kind), None, 0, ctypes.byref(n)))
    out = (nh_row_copy * max(1, n.value))()
    _check(lib.nh_slab_plan(len(ny_local), arr, int(kind), out, n.value, ctypes.byref(n)))
    return [(c.src_slab, c.src_row, c.dst_slab, c.dst_row, [b for b in range(32) if c.comp_mask >> b & 1])
            for c in out[:n.value]]


def nh_slab_init(ctxs, stream=None):
    arr = (_VP * len(ctxs))(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    _check(load_library().nh_slab_init(arr, len(ctxs), _VP(stream or 0)))


def nh_slab_step(ctxs, n_lb_steps: int, stream=None):
    arr = (_VP * len(ctxs))(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    _check(load_library().nh_slab_step(arr, len(ctxs), int(n_lb_steps), _VP(stream or 0)))


def nh_batch_autotune(ctxs, stream=None) -> int:
    arr = (_VP * len(ctxs))(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    out = ctypes.c_int(-1)
    _check(load_library().nh_batch_autotune(arr, len(ctxs), _VP(stream or 0), ctypes.byref(out)))
    return int(out.value)


def nh_relax(ctx, n_fd_steps: int, stream=None):
    _check(load_library().nh_relax(ctx, int(n_fd_steps), _VP(stream or 0)), ctx)


def nh_director_change(ctx) -> float:
    out = ctypes.c_double(0.0)
    _check(load_library().nh_director_change(ctx, ctypes.byref(out)), ctx)
    return float(out.value)


def nh_symmetrize_c4(ctx):
    _check(load_library().nh_symmetrize_c4(ctx), ctx)


def nh_batch_relax(ctxs, n_fd_steps: int, stream=None):
    arr = (_VP * len(ctxs))(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    _check(load_library().nh_batch_relax(arr, len(ctxs), int(n_fd_steps), _VP(stream or 0)))


def nh_set_solid(ctx, mask):
    """mask: host array [N] (1 = solid node), a CUDA uint8 tensor, or None."""
    if mask is None:
        _check(load_library().nh_set_solid(ctx, None, 0), ctx)
        return
    if hasattr(mask, "data_ptr"):
        _check(load_library().nh_set_solid(ctx, _VP(mask.data_ptr()), 1), ctx)
        return
    m = np.ascontiguousarray(np.asarray(mask).reshape(-1), dtype=np.uint8)
    _check(load_library().nh_set_solid(ctx, m.ctypes.data_as(_VP), 0), ctx)


def nh_set_tubes(ctx, centres):
    c = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1))
    _check(load_library().nh_set_tubes(ctx, c.ctypes.data_as(_DP), len(c) // 2), ctx)


def nh_diagnostics_enqueue(ctx, stream=None):
    _check(load_library().nh_diagnostics_enqueue(ctx, _VP(stream or 0)), ctx)


def nh_diagnostics_read(ctx, allow_unstable=False) -> dict:
    d = nh_diag()
    code = load_library().nh_diagnostics_read(ctx, ctypes.byref(d))
    return _diag_dict(ctx, d, code, allow_unstable)


def nh_diagnostics(ctx, allow_unstable=False) -> dict:
    d = nh_diag()
    code = load_library().nh_diagnostics(ctx, ctypes.byref(d))
    return _diag_dict(ctx, d, code, allow_unstable)


def _diag_dict(ctx, d, code, allow_unstable):
    if code != NH_OK and not (allow_unstable and code == NH_EUNSTABLE):
        _check(code, ctx)
    T = d.n_tubes
    return dict(step=d.step, mass=d.mass, energy=d.energy, max_u=d.max_u, min_norm=d.min_norm,
                max_norm=d.max_norm, nonfinite=d.nonfinite,
                centroids=np.array([[d.centroid[k][0], d.centroid[k][1]] for k in range(T)]).reshape(-1, 2),
                tube_weight=np.array([d.tube_weight[k] for k in range(T)]), code=code)


def nh_set_timing(ctx, mode):
    """0 = off, 1 (or True) = every kernel class, 2 = the LB class only."""
    _check(load_library().nh_set_timing(ctx, int(mode)), ctx)


def nh_get_timing(ctx) -> dict:
    t = nh_timing()
    _check(load_library().nh_get_timing(ctx, ctypes.byref(t)), ctx)
    return {k: (int(t.launches[i]), float(t.ms[i])) for i, k in enumerate(KCLASSES)}


def nh_launch_count(ctx) -> int:
    return int(load_library().nh_launch_count(ctx))


def nh_set_graphs(ctx, on: bool):
    _check(load_library().nh_set_graphs(ctx, 1 if on else 0), ctx)


def nh_set_wait_limit(ctx, seconds):
    _check(load_library().nh_set_wait_limit(ctx, float(seconds)), ctx)


def nh_set_diag_fold(ctx, on: bool):
    _check(load_library().nh_set_diag_fold(ctx, 1 if on else 0), ctx)


def nh_set_lb_variant(ctx, variant: int):
    _check(load_library().nh_set_lb_variant(ctx, int(variant)), ctx)


def nh_set_fd_variant(ctx, fused: int):
    _check(load_library().nh_set_fd_variant(ctx, int(fused)), ctx)


def nh_autotune(ctx, stream=None) -> int:
    out = ctypes.c_int(-1)
    _check(load_library().nh_autotune(ctx, _VP(stream or 0), ctypes.byref(out)), ctx)
    return int(out.value)


def nh_diagnostics_noalloc(p: nh_params, f, n, u, rho, out, stream=None):
    """Diagnostics from caller-owned device buffers (torch CUDA tensors) into
    out (a CUDA float64 tensor of 6); allocates no device memory."""
    _check(load_library().nh_diagnostics_noalloc(
        ctypes.byref(p), _VP(f.data_ptr()), _VP(n.data_ptr()), _VP(u.data_ptr()), _VP(rho.data_ptr()),
        _VP(out.data_ptr()), _VP(stream or 0)))


def nh_destroy(ctx):
    if ctx:
        load_library().nh_destroy(ctx)


# ------------------------------------------------------------------ convenience wrapper

class Channel:
    """One simulation channel: an nh context plus its torch-allocated workspace."""

    def __init__(self, params: dict, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the library has no CPU path")
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.params = dict(params)
        self.p = make_params(params)
        self.N = self.p.nx * self.p.ny * self.p.nz
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            nbytes = nh_workspace_bytes(self.p)
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) // 256 * 256
            self.ctx = nh_create(self.p, self.stream.cuda_stream)
            nh_bind_workspace(self.ctx, aligned, nbytes)
        self.workspace_bytes = nbytes

    # fields -------------------------------------------------------
    def set_fields(self, n, u=None, rho=None):
        if hasattr(n, "is_cuda") and n.is_cuda:
            nh_set_fields(self.ctx, n, u, rho, on_device=True)
            return
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        nh_set_fields(self.ctx, f(n), f(u), f(rho), on_device=False)

    def get_fields(self):
        n = np.empty((3, self.N))
        u = np.empty((3, self.N))
        rho = np.empty(self.N)
        nh_get_fields(self.ctx, n, u, rho)
        return n, u, rho

    def get_populations(self):
        f = np.empty((19, self.N))
        nh_get_populations(self.ctx, f)
        return f

    def set_populations(self, f):
        nh_set_populations(self.ctx, np.ascontiguousarray(f, dtype=np.float64))

    def get_force(self):
        F = np.empty((3, self.N))
        nh_get_force(self.ctx, F)
        return F

    def restore(self, n, F=None, u=None, rho=None, step=0):
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        nh_restore(self.ctx, f(n), f(F), f(u), f(rho), step)

    # stepping -----------------------------------------------------
    def step(self, count: int, stream=None):
        nh_step(self.ctx, count, (stream or self.stream).cuda_stream)

    def fd_update(self):
        nh_fd_update(self.ctx, self.stream.cuda_stream)

    def relax(self, n_fd_steps: int, stream=None):
        nh_relax(self.ctx, n_fd_steps, (stream or self.stream).cuda_stream)

    def symmetrize_c4(self):
        nh_symmetrize_c4(self.ctx)

    def director_change(self):
        return nh_director_change(self.ctx)

    def set_tubes(self, centres):
        nh_set_tubes(self.ctx, centres)

    def set_solid(self, mask):
        """Obstacle mask [N] (1 = solid node) or None; see nh_set_solid."""
        nh_set_solid(self.ctx, mask)

    def diagnostics(self, allow_unstable=False):
        return nh_diagnostics(self.ctx, allow_unstable)

    def diagnostics_enqueue(self, stream=None):
        nh_diagnostics_enqueue(self.ctx, (stream or self.stream).cuda_stream)

    def diagnostics_read(self, allow_unstable=False):
        return nh_diagnostics_read(self.ctx, allow_unstable)

    def set_timing(self, mode=1):
        nh_set_timing(self.ctx, mode)

    def timing(self):
        return nh_get_timing(self.ctx)

    def set_graphs(self, on=True):
        nh_set_graphs(self.ctx, on)

    def set_diag_fold(self, on=True):
        nh_set_diag_fold(self.ctx, on)

    def set_wait_limit(self, seconds):
        """Bound the host-side waits (seconds > 0; NHError with code NH_ETIMEOUT when exceeded)."""
        nh_set_wait_limit(self.ctx, seconds)

    def set_lb_variant(self, variant):
        nh_set_lb_variant(self.ctx, variant)

    def set_fd_variant(self, fused):
        nh_set_fd_variant(self.ctx, fused)

    def autotune(self):
        return nh_autotune(self.ctx, self.stream.cuda_stream)

    def launch_count(self):
        return nh_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            nh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_step(channels, n_lb_steps: int, stream=None):
    s = stream or channels[0].stream
    nh_batch_step([c.ctx for c in channels], n_lb_steps, s.cuda_stream)


def batch_relax(channels, n_fd_steps: int, stream=None):
    s = stream or channels[0].stream
    nh_batch_relax([c.ctx for c in channels], n_fd_steps, s.cuda_stream)


def batch_autotune(channels, stream=None) -> int:
    s = stream or channels[0].stream
    return nh_batch_autotune([c.ctx for c in channels], s.cuda_stream)


# ------------------------------------------------------------------ learned warm start network

def _dp(t):
    return None if t is None else _VP(t.data_ptr())


class UNet:
    """One warm-start network instance for a fixed (batch, nx, ny, nz); the FP32
    parameters (and Adam state) are shared torch CUDA tensors owned by the caller."""

    def __init__(self, batch, nx, ny, nz, device=0):
        import torch
        lib = load_library()
        self.torch = torch
        self.shape = (batch, nx, ny, nz)
        h = _VP()
        _check(lib.nh_unet_create(batch, nx, ny, nz, ctypes.byref(h)))
        self.h = h
        nb = ctypes.c_size_t(0)
        _check(lib.nh_unet_workspace_bytes(h, ctypes.byref(nb)))
        self.workspace = torch.empty(nb.value + 256, dtype=torch.uint8, device=torch.device("cuda", device))
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        _check(lib.nh_unet_bind(h, _VP(base), nb.value))

    @staticmethod
    def param_count():
        return int(load_library().nh_unet_param_count())

    def set_params(self, params, stream=None):
        _check(load_library().nh_unet_set_params(self.h, _dp(params), _VP(stream or 0)))

    def forward(self, params, n_ansatz, scalars, n_out=None, stream=None):
        _check(load_library().nh_unet_forward(self.h, _dp(params), _dp(n_ansatz), _dp(scalars), _dp(n_out),
                                              _VP(stream or 0)))

    def backward(self, params, n_ansatz, target, grad, loss, stream=None):
        _check(load_library().nh_unet_backward(self.h, _dp(params), _dp(n_ansatz), _dp(target), _dp(grad),
                                               _dp(loss), _VP(stream or 0)))

    def status(self, stream=None):
        """NHError (NH_ETIMEOUT) if a tensor-core convolution gave up a wait since the last check."""
        _check(load_library().nh_unet_status(self.h, _VP(stream or 0)))

    def activation(self, layer, out, stream=None):
        _check(load_library().nh_unet_activation(self.h, int(layer), _dp(out), _VP(stream or 0)))

    def close(self):
        if getattr(self, "h", None):
            load_library().nh_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nh_unet_adam(params, grad, m, v, step, lr, stream=None):
    _check(load_library().nh_unet_adam(_dp(params), _dp(grad), _dp(m), _dp(v), params.numel(), int(step),
                                       float(lr), _VP(stream or 0)))


class SlabGroup:
    """One channel split along y into slabs (nh_slab_*): slab k is a Channel
    over ny_local[k] interior rows plus a ghost row on each side.  Fields are
    split into and gathered from the slabs by indexing only."""

    def __init__(self, params: dict, ny_local, device: int = 0, stream=None):
        self.params = dict(params)
        self.ny_local = [int(v) for v in ny_local]
        assert sum(self.ny_local) == int(params["ny"]), "the slabs must cover the channel"
        self.y0 = np.concatenate([[0], np.cumsum(self.ny_local)[:-1]]).astype(int)
        self.slabs = [Channel(dict(params, ny=n + 2), device=device, stream=stream) for n in self.ny_local]
        self.stream = self.slabs[0].stream
        for ch in self.slabs:
            ch.set_fd_variant(0)

    def _rows(self, k):
        return (self.y0[k] - 1 + np.arange(self.ny_local[k] + 2)) % int(self.params["ny"])

    def _split(self, a, k, comps):
        if a is None:
            return None
        nx, ny, nz = int(self.params["nx"]), int(self.params["ny"]), int(self.params["nz"])
        g = np.asarray(a, dtype=np.float64).reshape(comps, nz, ny, nx)
        return np.ascontiguousarray(g[:, :, self._rows(k), :].reshape(comps, -1))

    def set_fields(self, n, u=None, rho=None):
        for k, ch in enumerate(self.slabs):
            r = self._split(rho, k, 1)
            ch.set_fields(self._split(n, k, 3), self._split(u, k, 3), None if r is None else r[0])
        nh_slab_init([c.ctx for c in self.slabs], self.stream.cuda_stream)

    def step(self, count: int):
        nh_slab_step([c.ctx for c in self.slabs], count, self.stream.cuda_stream)

    def _gather(self, parts, comps):
        nx, ny, nz = int(self.params["nx"]), int(self.params["ny"]), int(self.params["nz"])
        out = np.empty((comps, nz, ny, nx))
        for k, a in enumerate(parts):
            a = a.reshape(comps, nz, self.ny_local[k] + 2, nx)
            out[:, :, self.y0[k]:self.y0[k] + self.ny_local[k], :] = a[:, :, 1:-1, :]
        return out.reshape(comps, -1)

    def get_fields(self):
        got = [ch.get_fields() for ch in self.slabs]
        return (self._gather([g[0] for g in got], 3), self._gather([g[1] for g in got], 3),
                self._gather([g[2][None] for g in got], 1)[0])

    def get_populations(self):
        return self._gather([ch.get_populations() for ch in self.slabs], 19)

    def get_force(self):
        return self._gather([ch.get_force() for ch in self.slabs], 3)

    def close(self):
        for ch in self.slabs:
            ch.close()
