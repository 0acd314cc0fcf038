"""Python face of the FP64 CPU oracle of the DEM step (test infrastructure
only: the tests may import it, nothing in the product does).

Loads ``dem_oracle.c`` (gcc, ``-O2 -ffp-contract=off``) through ctypes.  The
contact model, the readings and the integration scheme are stated at the top
of that file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdemoracle.so")
_lock = threading.Lock()
_lib = None

# material and box parameters, in the order of the C prm[20] array
PARAM_KEYS = ("rho_p", "youngs", "poisson", "restitution", "friction", "rolling_friction",
              "wall_youngs", "wall_poisson", "wall_restitution", "wall_friction",
              "wall_rolling_friction")


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
            "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stdout=subprocess.DEVNULL,
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_dem_step.argtypes = [C.c_int64, dp, C.c_double, C.c_int, dp, dp, dp, dp, dp,
                                      dp, dp, C.c_int, C.POINTER(C.c_int32), dp, dp,
                                      C.POINTER(C.c_int)]
            L.or_dem_step.restype = C.c_int
            _lib = L
    return _lib


def params_array(p: dict) -> np.ndarray:
    a = [float(p[k]) for k in PARAM_KEYS]
    a += list(map(float, p.get("g", (0.0, 0.0, -9.81))))
    a += list(map(float, p["lo"])) + list(map(float, p["hi"]))
    return np.asarray(a, dtype=np.float64)


class State:
    """Particle state and contact memory of the oracle's DEM."""

    def __init__(self, x, v, w, r, capacity=24):
        self.x = np.ascontiguousarray(x, dtype=np.float64).copy()
        self.v = np.ascontiguousarray(v, dtype=np.float64).copy()
        self.w = np.ascontiguousarray(w, dtype=np.float64).copy()
        self.r = np.ascontiguousarray(r, dtype=np.float64).copy()
        n = self.x.shape[0]
        self.C = int(capacity)
        self.acc = np.zeros((n, 3))
        self.alpha = np.zeros((n, 3))
        self.hist_j = np.full(n * self.C, -1, dtype=np.int32)
        self.hist_t = np.zeros(n * self.C * 3)
        self.whist = np.zeros(n * 6 * 3)
        self.have_acc = C.c_int(0)

    def step(self, prm: dict, dt: float, nsub: int, f_ext=None):
        n = self.x.shape[0]
        fe = np.zeros((n, 3)) if f_ext is None else np.ascontiguousarray(f_ext, np.float64)
        pa = params_array(prm)
        dp = C.POINTER(C.c_double)
        st = lib().or_dem_step(n, pa.ctypes.data_as(dp), float(dt), int(nsub),
                               self.x.ctypes.data_as(dp), self.v.ctypes.data_as(dp),
                               self.w.ctypes.data_as(dp), self.r.ctypes.data_as(dp),
                               fe.ctypes.data_as(dp), self.acc.ctypes.data_as(dp),
                               self.alpha.ctypes.data_as(dp), self.C,
                               self.hist_j.ctypes.data_as(C.POINTER(C.c_int32)),
                               self.hist_t.ctypes.data_as(dp), self.whist.ctypes.data_as(dp),
                               C.byref(self.have_acc))
        return st


def glass_params(lo, hi, **over):
    """Glass beads in a glass box (Young's modulus reduced, as DEM codes do, to
    allow a practical time step)."""
    p = dict(rho_p=2500.0, youngs=1e7, poisson=0.3, restitution=0.9, friction=0.3,
             rolling_friction=0.0, wall_youngs=1e7, wall_poisson=0.3, wall_restitution=0.9,
             wall_friction=0.3, wall_rolling_friction=0.0, g=(0.0, 0.0, -9.81),
             lo=tuple(lo), hi=tuple(hi))
    p.update(over)
    return p
