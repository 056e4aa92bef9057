"""COSEnu oracle: plain FP64 CPU solver, used as test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product.

The arithmetic lives in ``cosenu_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so every rounding is the one written).  This module
compiles it on first use and exposes each entry point on numpy arrays.
Each function cites the passage of arXiv:2203.12866 it follows in the C file.

``OracleLib(path)`` wraps any build of the C file (the mutation tests load
deliberately broken copies); the module-level functions use the default build.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "cosenu_oracle.c")
_HDR = os.path.join(_HERE, "cosenu_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcosenu_oracle.so")

FDKO, WENO7, FDKO3 = 0, 1, 2
_lock = threading.Lock()
_default = None


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int64),
        ("nv", ctypes.c_int32),
        ("L", ctypes.c_double),
        ("scheme", ctypes.c_int32),
        ("hmode", ctypes.c_int32),
        ("mu", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("ko_eps", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("vgrid", ctypes.c_int32),
    ]


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp -ffp-contract=off of one oracle source into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           f"-I{_HERE}", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(SOURCE), os.path.getmtime(_HDR))
    if fresh and not force:
        return _LIB
    return compile_source(SOURCE, _LIB)


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


MIDPOINT, TRAPEZOID, SIMPSON = 0, 1, 2


def params(nz, nv, L, scheme=FDKO, *, mu=1.0, omega=0.0, theta=0.0, lam=0.0, ko_eps=0.1,
           weno_eps=1e-6, dt=None, cfl=0.4, hmode=1, vgrid=MIDPOINT) -> OracleParams:
    """Parameters of one run.  dt defaults to cfl * dz with max|v| taken as 1."""
    if dt is None:
        dt = cfl * L / nz
    return OracleParams(int(nz), int(nv), float(L), int(scheme), int(hmode), float(mu),
                        float(omega), float(theta), float(lam), float(ko_eps), float(weno_eps),
                        float(dt), int(vgrid))


class OracleLib:
    """The oracle's entry points on numpy arrays, bound to one compiled library."""

    FDKO, WENO7, FDKO3 = FDKO, WENO7, FDKO3
    MIDPOINT, TRAPEZOID, SIMPSON = 0, 1, 2
    params = staticmethod(params)

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        pp = P(OracleParams)
        lib.oracle_vgrid.argtypes = [ctypes.c_int32, dp, dp]
        lib.oracle_vgrid_q.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp]
        lib.oracle_hamiltonian.argtypes = [pp, dp, dp]
        lib.oracle_rhs.argtypes = [pp, dp, dp]
        lib.oracle_step.argtypes = [pp, dp, ctypes.c_int64]
        lib.oracle_weno7_face.argtypes = [dp, ctypes.c_double, dp]
        lib.oracle_weno7_face.restype = ctypes.c_double
        lib.oracle_conserved.argtypes = [pp, dp, dp]
        lib.oracle_moments.argtypes = [pp, dp, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _state(p, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == 8 * p.nz * p.nv, "state must be [2][4][nz][nv]"
        return u

    def vgrid(self, nv, mode=MIDPOINT):
        v = np.empty(nv)
        w = np.empty(nv)
        if mode == MIDPOINT:
            self.lib.oracle_vgrid(nv, _ptr(v), _ptr(w))
        else:
            assert self.lib.oracle_vgrid_q(nv, int(mode), _ptr(v), _ptr(w)) == 0
        return v, w

    def hamiltonian(self, p, u):
        u = self._state(p, u)
        out = np.empty((2, 3, p.nz, p.nv))
        assert self.lib.oracle_hamiltonian(ctypes.byref(p), _ptr(u), _ptr(out)) == 0
        return out

    def rhs(self, p, u):
        u = self._state(p, u)
        k = np.empty_like(u)
        assert self.lib.oracle_rhs(ctypes.byref(p), _ptr(u), _ptr(k)) == 0
        return k

    def step(self, p, y, nsteps=1):
        """Return y advanced by nsteps RK4 steps (the input is not modified)."""
        y = self._state(p, y).copy()
        assert self.lib.oracle_step(ctypes.byref(p), _ptr(y), int(nsteps)) == 0
        return y

    def weno7_face(self, f, eps=1e-6, detail=False):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == 7
        d = np.empty(12)
        val = self.lib.oracle_weno7_face(_ptr(f), float(eps), _ptr(d))
        if detail:
            return val, {"f4": d[0:4].copy(), "si": d[4:8].copy(), "wbar": d[8:12].copy()}
        return val

    def conserved(self, p, u):
        """dict: tr_nu, tr_nubar, M (3,), M_vac, dP_max, dP_mean."""
        u = self._state(p, u)
        out = np.empty(10)
        assert self.lib.oracle_conserved(ctypes.byref(p), _ptr(u), _ptr(out)) == 0
        return {"tr_nu": out[0], "tr_nubar": out[1], "M": out[2:5].copy(), "M_vac": out[5],
                "dP_max": out[6], "dP_mean": out[7]}

    def moments(self, p, u):
        """(zavg [2][4][nv], vmom [nz][6])."""
        u = self._state(p, u)
        zavg = np.empty((2, 4, p.nv))
        vmom = np.empty((p.nz, 6))
        assert self.lib.oracle_moments(ctypes.byref(p), _ptr(u), _ptr(zavg), _ptr(vmom)) == 0
        return zavg, vmom

    def num_threads(self):
        return int(self.lib.oracle_num_threads())


def _lib() -> OracleLib:
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
    return _default


def vgrid(nv, mode=MIDPOINT):
    return _lib().vgrid(nv, mode)


def hamiltonian(p, u):
    return _lib().hamiltonian(p, u)


def rhs(p, u):
    return _lib().rhs(p, u)


def step(p, y, nsteps=1):
    return _lib().step(p, y, nsteps)


def weno7_face(f, eps=1e-6, detail=False):
    return _lib().weno7_face(f, eps, detail)


def conserved(p, u):
    return _lib().conserved(p, u)


def moments(p, u):
    return _lib().moments(p, u)


def num_threads():
    return _lib().num_threads()
