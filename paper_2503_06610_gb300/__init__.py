"""GB300 (sm_103a) hybrid lattice-Boltzmann + finite-difference nematohydrodynamics.

The method is arXiv:2503.06610 ("Efficient single-precision simulations of
nematohydrodynamics"): D3Q19 LB with shifted populations and Guo forcing for
the flow, an Ericksen-Leslie director advanced by a predictor-corrector on its
own time step dt_FD, coupled through the LC stress divergence.

* ``nh``      - ctypes binding of the C ABI (``include/nh.h``) and ``Channel``;
* ``inputs``  - seeded synthetic initial conditions and parameter presets;
* ``build``   - nvcc build of the CUDA library into ``_lib/libnh.so``.

The CUDA library does every computation; importing this package does not load
it (``nh.load_library()`` does, on first use).
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "nh", "build"]


def __getattr__(name):
    if name in ("nh", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
