"""GB300-native EXCMG solver for the 3D biharmonic equation with the 25-point
scheme (Pan, He & Ni, arXiv 1901.05118).

The solver is the CUDA library ``libexcmg.so`` (C ABI: ``include/excmg.h``);
this package exposes it through a thin ctypes binding with the same names.
``problems`` holds the seeded manufactured inputs.  The binding is loaded on
first use of an API name, and raises if the library has not been built.
"""
_API = ("excmg_solve", "stencil_apply", "bicg_solve", "extrapolate_interpolate", "midpoint_extrapolate",
        "excmg_assemble_rhs", "excmg_dsolve", "Context", "Level", "ExcmgError", "default_context", "Batch")

__all__ = list(_API) + ["problems"]


def __getattr__(name):
    if name in _API:
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
