"""GB300-native split-step Crank-Nicolson solver of the 3D Gross-Pitaevskii
equation in a fully anisotropic harmonic trap (imaginary and real time).

The hot path (kick, CN line solves along x, y and z, renormalisation and the
observables reductions) runs in hand-written CUDA kernels for sm_103a inside
libgpcn.so, behind the C ABI declared in include/gp.h.  This package holds
the build script, the ctypes binding and a thin PyTorch-backed front end.
"""
from . import inputs  # noqa: F401  (seeded synthetic workloads, no method arithmetic)

__all__ = ["GP", "build", "inputs"]


def __getattr__(name):
    if name == "GP":
        from .solver import GP
        return GP
    if name == "build":
        import importlib
        return importlib.import_module(__name__ + ".build")
    raise AttributeError(name)
