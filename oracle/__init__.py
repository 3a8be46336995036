"""FP64 CPU oracle of the binary Shan-Chen D2Q9 capillary step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product library never does:
this is the checker, independent of the CUDA path (no shared code, headers or
constants).  The arithmetic lives in ``shanchen_oracle.c`` (plain loops, FP64,
no FMA contraction); this module only marshals numpy arrays through ctypes.

Paper: S. Chibbaro, "Capillary filling with pseudo-potential binary
Lattice-Boltzmann model", Model section (Eqs. 2-11) and Numerical Results
section (geometry, bounce-back, interface and precursor fronts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shanchen_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, ``-ffp-contract=off``)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("cap_x0", ctypes.c_int32), ("cap_x1", ctypes.c_int32),
        ("y_bot", ctypes.c_int32), ("y_top", ctypes.c_int32),
        ("G", ctypes.c_double), ("Gw", ctypes.c_double * 2),
        ("tau", ctypes.c_double * 2), ("body", ctypes.c_double * 2),
        ("rho_bulk", ctypes.c_double),
        ("alpha", ctypes.c_double * 2), ("mass", ctypes.c_double * 2),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            lib.oc_create.restype = ctypes.c_void_p
            lib.oc_create.argtypes = [P(_Params), P(ctypes.c_uint8), dp, dp]
            lib.oc_destroy.argtypes = [ctypes.c_void_p]
            lib.oc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.oc_time.restype = ctypes.c_long
            lib.oc_time.argtypes = [ctypes.c_void_p]
            lib.oc_stream.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oc_collide.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oc_get_populations.argtypes = [ctypes.c_void_p, dp]
            lib.oc_set_populations.argtypes = [ctypes.c_void_p, dp]
            lib.oc_get_solid.argtypes = [ctypes.c_void_p, P(ctypes.c_uint8)]
            lib.oc_densities.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oc_accel.argtypes = [ctypes.c_void_p, dp, dp, dp]
            lib.oc_velocity.restype = ctypes.c_int
            lib.oc_velocity.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oc_mass.argtypes = [ctypes.c_void_p, dp]
            lib.oc_momentum.argtypes = [ctypes.c_void_p, dp]
            lib.oc_interface.restype = ctypes.c_int
            lib.oc_interface.argtypes = [ctypes.c_void_p, dp]
            lib.oc_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            lib.oc_feq_alpha.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            lib.oc_pressure_general.restype = ctypes.c_double
            lib.oc_pressure_general.argtypes = [ctypes.c_double] * 7
            lib.oc_pressure.restype = ctypes.c_double
            lib.oc_pressure.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def feq(n: float, ux: float, uy: float, alpha: float = 4.0 / 9.0) -> np.ndarray:
    """Eqs. 3-5 for one node: the 9 equilibrium populations."""
    out = np.zeros(9)
    _load().oc_feq_alpha(float(n), float(ux), float(uy), float(alpha), _dp(out))
    return out


def pressure(nA, nB, G: float, alpha=(4.0 / 9.0, 4.0 / 9.0), mass=(1.0, 1.0)):
    """Mixture pressure p = m_A cA n_A + m_B cB n_B + G n_A n_B / 3 with
    c^2 = 3 (1 - alpha) / 5 (Model section); (n_A + n_B)/3 + G n_A n_B / 3 at
    alpha = 4/9, m = 1."""
    lib = _load()
    if tuple(alpha) == (4.0 / 9.0, 4.0 / 9.0) and tuple(mass) == (1.0, 1.0):
        f = np.vectorize(lambda a, b: lib.oc_pressure(float(a), float(b), float(G)))
    else:
        f = np.vectorize(lambda a, b: lib.oc_pressure_general(float(a), float(b), float(G), float(alpha[0]),
                                                              float(alpha[1]), float(mass[0]), float(mass[1])))
    return f(nA, nB)


class OracleLattice:
    """One capillary run on the CPU in FP64.

    ``geom`` keys: nx, ny, cap_x0, cap_x1, y_bot, y_top (-1 = none), optional
    ``mask`` (uint8 [ny, nx]).  ``params`` keys: G, G_Aw, G_Bw, tau_A, tau_B,
    optional body (gx, gy), rho_bulk, alpha (2-tuple, Eqs. 3-5, default 4/9)
    and mass (2-tuple of molecular masses, default 1).  ``nA0``/``nB0`` are the initial
    densities ([ny, nx]); the state starts at rest in equilibrium.
    """

    def __init__(self, geom: dict, params: dict, nA0: np.ndarray, nB0: np.ndarray):
        lib = _load()
        self.nx, self.ny = int(geom["nx"]), int(geom["ny"])
        p = _Params()
        p.nx, p.ny = self.nx, self.ny
        p.cap_x0, p.cap_x1 = int(geom.get("cap_x0", 0)), int(geom.get("cap_x1", 0))
        p.y_bot, p.y_top = int(geom.get("y_bot", -1)), int(geom.get("y_top", -1))
        p.G = float(params["G"])
        p.Gw[0], p.Gw[1] = float(params.get("G_Aw", 0.0)), float(params.get("G_Bw", 0.0))
        p.tau[0], p.tau[1] = float(params["tau_A"]), float(params["tau_B"])
        body = params.get("body", (0.0, 0.0))
        p.body[0], p.body[1] = float(body[0]), float(body[1])
        p.rho_bulk = float(params.get("rho_bulk", 2.0))
        alpha = params.get("alpha", (4.0 / 9.0, 4.0 / 9.0))
        mass = params.get("mass", (1.0, 1.0))
        p.alpha[0], p.alpha[1] = float(alpha[0]), float(alpha[1])
        p.mass[0], p.mass[1] = float(mass[0]), float(mass[1])
        self._p = p
        shape = (self.ny, self.nx)
        nA0 = np.ascontiguousarray(nA0, dtype=np.float64).reshape(shape)
        nB0 = np.ascontiguousarray(nB0, dtype=np.float64).reshape(shape)
        mask = geom.get("mask")
        mptr = None
        if mask is not None:
            self._mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(shape)
            mptr = self._mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        h = lib.oc_create(ctypes.byref(p), mptr, _dp(nA0), _dp(nB0))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.oc_destroy(h)
            self._h = None

    @property
    def t(self) -> int:
        return int(self._lib.oc_time(self._h))

    @property
    def N(self) -> int:
        return self.nx * self.ny

    def step(self, n: int = 1) -> None:
        self._lib.oc_step(self._h, int(n))

    def populations(self) -> np.ndarray:
        """Post-collision populations, shape [2, 9, ny, nx]."""
        F = np.zeros((2, 9, self.ny, self.nx))
        self._lib.oc_get_populations(self._h, _dp(F))
        return F

    def set_populations(self, F: np.ndarray) -> None:
        F = np.ascontiguousarray(F, dtype=np.float64).reshape(2, 9, self.ny, self.nx)
        self._lib.oc_set_populations(self._h, _dp(F))

    def solid(self) -> np.ndarray:
        s = np.zeros((self.ny, self.nx), dtype=np.uint8)
        self._lib.oc_get_solid(self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return s

    def stream(self, F: np.ndarray) -> np.ndarray:
        """Streaming with bounce-back only (left-hand side of Eq. 2)."""
        F = np.ascontiguousarray(F, dtype=np.float64).reshape(2, 9, self.ny, self.nx)
        out = np.zeros_like(F)
        self._lib.oc_stream(self._h, _dp(F), _dp(out))
        return out

    def collide(self, ft: np.ndarray) -> np.ndarray:
        """Collision alone (right-hand side of Eq. 2) of streamed populations."""
        ft = np.ascontiguousarray(ft, dtype=np.float64).reshape(2, 9, self.ny, self.nx)
        out = np.zeros_like(ft)
        self._lib.oc_collide(self._h, _dp(ft), _dp(out))
        return out

    def densities(self):
        nA = np.zeros((self.ny, self.nx))
        nB = np.zeros((self.ny, self.nx))
        self._lib.oc_densities(self._h, _dp(nA), _dp(nB))
        return nA, nB

    def accel(self, nA: np.ndarray, nB: np.ndarray) -> np.ndarray:
        """Accelerations [aAx, aAy, aBx, aBy] for given density fields (Eqs. 9-11)."""
        nA = np.ascontiguousarray(nA, dtype=np.float64).reshape(self.ny, self.nx)
        nB = np.ascontiguousarray(nB, dtype=np.float64).reshape(self.ny, self.nx)
        out = np.zeros((4, self.ny, self.nx))
        self._lib.oc_accel(self._h, _dp(nA), _dp(nB), _dp(out))
        return out

    def velocity(self):
        ux = np.zeros((self.ny, self.nx))
        uy = np.zeros((self.ny, self.nx))
        self._lib.oc_velocity(self._h, _dp(ux), _dp(uy))
        return ux, uy

    def mass(self) -> np.ndarray:
        M = np.zeros(2)
        self._lib.oc_mass(self._h, _dp(M))
        return M

    def momentum(self) -> np.ndarray:
        P = np.zeros(2)
        self._lib.oc_momentum(self._h, _dp(P))
        return P

    def interface(self) -> np.ndarray:
        """[z_bulk, z_prec_bottom, z_prec_top] measured from cap_x0."""
        out = np.zeros(3)
        self._lib.oc_interface(self._h, _dp(out))
        return out
