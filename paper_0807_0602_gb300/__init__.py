"""GB300-native binary Shan-Chen D2Q9 capillary-filling library.

The method (S. Chibbaro, "Capillary filling with pseudo-potential binary
Lattice-Boltzmann model"): two immiscible components, per-component BGK with
the equilibrium-velocity shift, cross-species pseudo-potential force, wall
force setting the contact angle, half-way bounce-back on the plates, and the
bulk-interface and precursor-film fronts z(t); species with the standard
D2Q9 equilibrium or with a free rest fraction alpha_k and molecular mass m_k
(density ratios).  The step runs in hand-written CUDA kernels for sm_103a
behind the C ABI of include/lbm.h; this package holds the Python binding
(``Lattice``), the host-side analysis and the build step.
"""
from .build import build as build_library  # noqa: F401


def __getattr__(name):
    if name in ("Lattice", "LbmError"):
        from . import lbm, _lib
        return {"Lattice": lbm.Lattice, "LbmError": _lib.LbmError}[name]
    raise AttributeError(name)
