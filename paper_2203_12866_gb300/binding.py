"""Thin ctypes binding of libcosenu.so (include/cosenu.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions keep the C names; ``Solver`` is a small convenience
owner of one handle.  If the library is missing, loading raises -- there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcosenu.so")

COSENU_FDKO, COSENU_WENO7, COSENU_FDKO3 = 0, 1, 2
COSENU_FP64, COSENU_MIXED = 0, 1
COSENU_OK, COSENU_EINVAL, COSENU_ENOMEM, COSENU_ECUDA, COSENU_ENONFINITE, COSENU_ETIMEOUT = (
    0, -1, -2, -3, -4, -5)
COSENU_ECANCELLED, COSENU_PENDING = -6, 1
COSENU_MIDPOINT, COSENU_TRAPEZOID, COSENU_SIMPSON = 0, 1, 2

# Every entry point include/cosenu.h declares.
EXPORTS = (
    "cosenu_create", "cosenu_workspace_bytes", "cosenu_create_external", "cosenu_destroy",
    "cosenu_set_quadrature", "cosenu_velocities", "cosenu_set_params", "cosenu_get_params",
    "cosenu_set_stream", "cosenu_set_state", "cosenu_set_state_device",
    "cosenu_set_state_collective", "cosenu_get_state", "cosenu_get_rows", "cosenu_state_device",
    "cosenu_step", "cosenu_sync", "cosenu_moments", "cosenu_running_moments", "cosenu_conserved",
    "cosenu_dp_field", "cosenu_spectrum", "cosenu_set_stage_timing", "cosenu_stage_times",
    "cosenu_steps_taken", "cosenu_last_error", "cosenu_kernel_launches", "cosenu_batch_create", "cosenu_batch_destroy",
    "cosenu_batch_add", "cosenu_batch_remove", "cosenu_batch_size", "cosenu_batch_device_bytes",
    "cosenu_batch_step", "cosenu_batch_sync", "cosenu_batch_member", "cosenu_batch_tune",
    "cosenu_batch_classes", "cosenu_batch_class_info", "cosenu_batch_set_stage_timing",
    "cosenu_batch_stage_times", "cosenu_batch_stream", "cosenu_batch_last_error",
    "cosenu_server_create", "cosenu_server_destroy", "cosenu_submit", "cosenu_poll", "cosenu_wait",
    "cosenu_cancel", "cosenu_server_get_stats", "cosenu_server_last_error",
    "cosenu_conserved_noalloc",
)


class cosenu_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("mu", "omega", "theta", "lambda_", "ko_eps", "weno_eps", "dt")]


class cosenu_conserved_t(ctypes.Structure):
    _fields_ = [("tr_nu", ctypes.c_double), ("tr_nubar", ctypes.c_double),
                ("M", ctypes.c_double * 3), ("M_vac", ctypes.c_double),
                ("dP_max", ctypes.c_double), ("dP_mean", ctypes.c_double),
                ("step", ctypes.c_int64)]


class cosenu_batch_class(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nv", ctypes.c_int32), ("members", ctypes.c_int32), ("rows", ctypes.c_int64),
                ("rows_per_slot", ctypes.c_int32 * 4), ("ring", ctypes.c_int32 * 4),
                ("grid", ctypes.c_int32 * 4), ("smem", ctypes.c_int32 * 4),
                ("occupancy", ctypes.c_int32 * 4), ("concurrent", ctypes.c_int32),
                ("kernel_ms", ctypes.c_double * 5)]


class cosenu_request(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int64), ("nv", ctypes.c_int32), ("L", ctypes.c_double),
                ("scheme", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("params", cosenu_params), ("nsteps", ctypes.c_int64),
                ("state", ctypes.POINTER(ctypes.c_double)), ("alpha", ctypes.c_double),
                ("sigma_nu", ctypes.c_double), ("sigma_nubar", ctypes.c_double),
                ("eps0", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("out_state", ctypes.POINTER(ctypes.c_double))]


class cosenu_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("conserved", cosenu_conserved_t), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class cosenu_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("finished", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("queued", ctypes.c_int32),
                ("running", ctypes.c_int32), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("budget", ctypes.c_size_t)]


class CosenuError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cosenu error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libcosenu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2203_12866_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    i64, i32, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
    sig = {
        "cosenu_create": (vp, [i64, i32, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
        "cosenu_workspace_bytes": (sz, [i64, i32, ctypes.c_int, ctypes.c_int]),
        "cosenu_create_external": (vp, [i64, i32, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        vp, sz]),
        "cosenu_destroy": (None, [vp]),
        "cosenu_set_quadrature": (ctypes.c_int, [vp, i32]),
        "cosenu_velocities": (ctypes.c_int, [vp, dp, dp]),
        "cosenu_set_params": (ctypes.c_int, [vp, ctypes.POINTER(cosenu_params)]),
        "cosenu_get_params": (ctypes.c_int, [vp, ctypes.POINTER(cosenu_params)]),
        "cosenu_set_stream": (ctypes.c_int, [vp, vp]),
        "cosenu_set_state": (ctypes.c_int, [vp, dp, sz]),
        "cosenu_set_state_device": (ctypes.c_int, [vp, vp, sz]),
        "cosenu_set_state_collective": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double,
                                                       ctypes.c_double, ctypes.c_double,
                                                       ctypes.c_uint64]),
        "cosenu_get_state": (ctypes.c_int, [vp, dp, sz]),
        "cosenu_get_rows": (ctypes.c_int, [vp, i64, i64, dp]),
        "cosenu_state_device": (vp, [vp]),
        "cosenu_step": (ctypes.c_int, [vp, i64]),
        "cosenu_sync": (ctypes.c_int, [vp]),
        "cosenu_moments": (ctypes.c_int, [vp, dp, dp]),
        "cosenu_running_moments": (ctypes.c_int, [vp, dp]),
        "cosenu_conserved": (ctypes.c_int, [vp, ctypes.POINTER(cosenu_conserved_t)]),
        "cosenu_dp_field": (ctypes.c_int, [vp, dp]),
        "cosenu_spectrum": (ctypes.c_int, [vp, i32, i32, i64, i64, dp]),
        "cosenu_set_stage_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "cosenu_stage_times": (ctypes.c_int, [vp, dp, ctypes.POINTER(i64)]),
        "cosenu_steps_taken": (i64, [vp]),
        "cosenu_last_error": (ctypes.c_char_p, [vp]),
        "cosenu_kernel_launches": (ctypes.c_uint64, []),
        "cosenu_conserved_noalloc": (ctypes.c_int, [vp, i64, i32, ctypes.c_double, ctypes.c_double,
                                                    vp, vp]),
        "cosenu_batch_create": (vp, []),
        "cosenu_batch_destroy": (None, [vp]),
        "cosenu_batch_add": (ctypes.c_int, [vp, i64, i32, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(vp)]),
        "cosenu_batch_remove": (ctypes.c_int, [vp, vp]),
        "cosenu_batch_size": (i32, [vp]),
        "cosenu_batch_device_bytes": (sz, [vp]),
        "cosenu_batch_step": (ctypes.c_int, [vp, i64]),
        "cosenu_batch_sync": (ctypes.c_int, [vp, ctypes.POINTER(i32)]),
        "cosenu_batch_member": (vp, [vp, i32]),
        "cosenu_batch_tune": (ctypes.c_int, [vp, i32, ctypes.POINTER(i64)]),
        "cosenu_batch_classes": (i32, [vp]),
        "cosenu_batch_class_info": (ctypes.c_int, [vp, i32, ctypes.POINTER(cosenu_batch_class)]),
        "cosenu_batch_set_stage_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "cosenu_batch_stage_times": (ctypes.c_int, [vp, dp, ctypes.POINTER(i64)]),
        "cosenu_batch_stream": (vp, [vp]),
        "cosenu_server_create": (vp, [sz, i32, i32]),
        "cosenu_server_destroy": (None, [vp]),
        "cosenu_submit": (ctypes.c_int, [vp, ctypes.POINTER(cosenu_request),
                                         ctypes.POINTER(ctypes.c_uint64)]),
        "cosenu_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(cosenu_result)]),
        "cosenu_wait": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.POINTER(cosenu_result)]),
        "cosenu_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "cosenu_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(cosenu_server_stats)]),
        "cosenu_server_last_error": (ctypes.c_char_p, [vp]),
        "cosenu_batch_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(h, rc):
    if rc != COSENU_OK:
        raise CosenuError(rc, load().cosenu_last_error(h).decode())
    return rc


# ---------------------------------------------------------------- C-named wrappers

def cosenu_create(nz, nv, L, scheme=COSENU_FDKO, precision=COSENU_FP64):
    lib = load()
    h = lib.cosenu_create(int(nz), int(nv), float(L), int(scheme), int(precision))
    if not h:
        raise CosenuError(COSENU_EINVAL, lib.cosenu_last_error(None).decode())
    return h


def cosenu_workspace_bytes(nz, nv, scheme=COSENU_FDKO, precision=COSENU_FP64):
    return int(load().cosenu_workspace_bytes(int(nz), int(nv), int(scheme), int(precision)))


def cosenu_create_external(nz, nv, L, scheme, precision, workspace_ptr, workspace_bytes):
    lib = load()
    h = lib.cosenu_create_external(int(nz), int(nv), float(L), int(scheme), int(precision),
                                   ctypes.c_void_p(int(workspace_ptr)), int(workspace_bytes))
    if not h:
        raise CosenuError(COSENU_EINVAL, lib.cosenu_last_error(None).decode())
    return h


def cosenu_destroy(h):
    load().cosenu_destroy(h)


def cosenu_set_quadrature(h, mode):
    return _check(h, load().cosenu_set_quadrature(h, int(mode)))


def cosenu_velocities(h, nv):
    v = np.empty(nv)
    w = np.empty(nv)
    _check(h, load().cosenu_velocities(h, _dptr(v), _dptr(w)))
    return v, w


def cosenu_set_params(h, **kw):
    p = cosenu_get_params(h)
    for k, v in kw.items():
        setattr(p, "lambda_" if k in ("lambda", "lam") else k, float(v))
    return _check(h, load().cosenu_set_params(h, ctypes.byref(p)))


def cosenu_get_params(h):
    p = cosenu_params()
    _check(h, load().cosenu_get_params(h, ctypes.byref(p)))
    return p


def cosenu_set_stream(h, stream_handle):
    return _check(h, load().cosenu_set_stream(h, ctypes.c_void_p(int(stream_handle or 0))))


def cosenu_set_state(h, host):
    a = np.ascontiguousarray(host, dtype=np.float64)
    return _check(h, load().cosenu_set_state(h, _dptr(a), a.size))


def cosenu_set_state_device(h, dev_ptr, n):
    return _check(h, load().cosenu_set_state_device(h, ctypes.c_void_p(int(dev_ptr)), int(n)))


def cosenu_set_state_collective(h, alpha=0.9, sigma_nu=0.6, sigma_nubar=0.5, eps0=1e-6,
                                seed=12866):
    return _check(h, load().cosenu_set_state_collective(h, float(alpha), float(sigma_nu),
                                                         float(sigma_nubar), float(eps0),
                                                         int(seed)))


def cosenu_get_state(h, out):
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    return _check(h, load().cosenu_get_state(h, _dptr(out), out.size))


def cosenu_get_rows(h, z0, nrows, out):
    assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
    return _check(h, load().cosenu_get_rows(h, int(z0), int(nrows), _dptr(out)))


def cosenu_state_device(h):
    return int(load().cosenu_state_device(h) or 0)


def cosenu_step(h, nsteps=1):
    return _check(h, load().cosenu_step(h, int(nsteps)))


def cosenu_sync(h):
    return _check(h, load().cosenu_sync(h))


def cosenu_moments(h, zavg=None, vmom=None):
    return _check(h, load().cosenu_moments(h, _dptr(zavg), _dptr(vmom)))


def cosenu_running_moments(h, nz):
    """The per-z moments [nz][6] the next stage kernel uses for H (see include/cosenu.h)."""
    out = np.empty((nz, 6))
    _check(h, load().cosenu_running_moments(h, _dptr(out)))
    return out


def cosenu_conserved(h):
    c = cosenu_conserved_t()
    _check(h, load().cosenu_conserved(h, ctypes.byref(c)))
    return {"tr_nu": c.tr_nu, "tr_nubar": c.tr_nubar, "M": np.array(c.M[:]), "M_vac": c.M_vac,
            "dP_max": c.dP_max, "dP_mean": c.dP_mean, "step": c.step}


def cosenu_dp_field(h, nz, nv):
    out = np.empty((2, nz, nv))
    _check(h, load().cosenu_dp_field(h, _dptr(out)))
    return out


def cosenu_spectrum(h, species, v_index, m0, nk):
    """Complex X(m) for m = m0 .. m0 + nk - 1 (see include/cosenu.h)."""
    out = np.empty(2 * int(nk))
    _check(h, load().cosenu_spectrum(h, int(species), int(v_index), int(m0), int(nk),
                                     _dptr(out)))
    return out[0::2] + 1j * out[1::2]


def cosenu_set_stage_timing(h, on=True):
    return _check(h, load().cosenu_set_stage_timing(h, 1 if on else 0))


def cosenu_stage_times(h):
    """(ms[5], launches[5]) summed per kernel of the step (stages 1-4, increment) since
    the last call."""
    ms = np.zeros(5)
    n = (ctypes.c_int64 * 5)()
    _check(h, load().cosenu_stage_times(h, _dptr(ms), n))
    return ms, np.array(n[:], dtype=np.int64)


def cosenu_steps_taken(h):
    return int(load().cosenu_steps_taken(h))


def cosenu_last_error(h=None):
    return load().cosenu_last_error(h).decode()


def cosenu_kernel_launches():
    return int(load().cosenu_kernel_launches())


def cosenu_conserved_noalloc(y_dev_ptr, nz, nv, L, theta, out_dev_ptr, stream_handle=0):
    """Enqueue the allocation-free diagnostics of a device state into a caller-owned
    device buffer of 8 doubles (see include/cosenu.h)."""
    rc = load().cosenu_conserved_noalloc(ctypes.c_void_p(int(y_dev_ptr)), int(nz), int(nv),
                                         float(L), float(theta), ctypes.c_void_p(int(out_dev_ptr)),
                                         ctypes.c_void_p(int(stream_handle or 0)))
    return _check(None, rc)


# ---------------------------------------------------------------- batched solver

def _bcheck(b, rc):
    if rc != COSENU_OK:
        raise CosenuError(rc, load().cosenu_batch_last_error(b).decode())
    return rc


def cosenu_batch_create():
    lib = load()
    b = lib.cosenu_batch_create()
    if not b:
        raise CosenuError(COSENU_ECUDA, lib.cosenu_batch_last_error(None).decode())
    return b


def cosenu_batch_destroy(b):
    load().cosenu_batch_destroy(b)


def cosenu_batch_add(b, nz, nv, L, scheme=COSENU_FDKO, precision=COSENU_MIXED):
    h = ctypes.c_void_p()
    _bcheck(b, load().cosenu_batch_add(b, int(nz), int(nv), float(L), int(scheme), int(precision),
                                       ctypes.byref(h)))
    return h.value


def cosenu_batch_remove(b, member):
    return _bcheck(b, load().cosenu_batch_remove(b, member))


def cosenu_batch_size(b):
    return int(load().cosenu_batch_size(b))


def cosenu_batch_device_bytes(b):
    return int(load().cosenu_batch_device_bytes(b))


def cosenu_batch_step(b, nsteps=1):
    return _bcheck(b, load().cosenu_batch_step(b, int(nsteps)))


def cosenu_batch_sync(b):
    """Returns (rc, first_bad) without raising on COSENU_ENONFINITE / COSENU_ETIMEOUT."""
    bad = ctypes.c_int32(-1)
    rc = load().cosenu_batch_sync(b, ctypes.byref(bad))
    if rc not in (COSENU_OK, COSENU_ENONFINITE, COSENU_ETIMEOUT):
        _bcheck(b, rc)
    return rc, int(bad.value)


def cosenu_batch_member(b, i):
    return load().cosenu_batch_member(b, int(i))


def cosenu_batch_tune(b, reps=2):
    """Run the autotuner; returns the number of steps the members advanced."""
    n = ctypes.c_int64(0)
    _bcheck(b, load().cosenu_batch_tune(b, int(reps), ctypes.byref(n)))
    return int(n.value)


def cosenu_batch_classes(b):
    n = int(load().cosenu_batch_classes(b))
    if n < 0:
        raise CosenuError(COSENU_ECUDA, load().cosenu_batch_last_error(b).decode())
    return n


def cosenu_batch_class_info(b, c):
    info = cosenu_batch_class()
    _bcheck(b, load().cosenu_batch_class_info(b, int(c), ctypes.byref(info)))
    return {"scheme": info.scheme, "precision": info.precision, "nv": info.nv,
            "members": info.members, "rows": info.rows,
            "rows_per_slot": list(info.rows_per_slot), "ring": list(info.ring),
            "grid": list(info.grid), "smem": list(info.smem),
            "occupancy": list(info.occupancy), "concurrent": bool(info.concurrent),
            "kernel_ms": list(info.kernel_ms)}


def cosenu_batch_set_stage_timing(b, on=True):
    return _bcheck(b, load().cosenu_batch_set_stage_timing(b, 1 if on else 0))


def cosenu_batch_stage_times(b):
    ms = np.zeros(5)
    n = (ctypes.c_int64 * 5)()
    _bcheck(b, load().cosenu_batch_stage_times(b, _dptr(ms), n))
    return ms, np.array(n[:], dtype=np.int64)


def cosenu_batch_stream(b):
    return int(load().cosenu_batch_stream(b) or 0)


def cosenu_batch_last_error(b=None):
    return load().cosenu_batch_last_error(b).decode()


# ---------------------------------------------------------------- serving

def _scheck(srv, rc):
    if rc < 0:
        raise CosenuError(rc, load().cosenu_server_last_error(srv).decode())
    return rc


def cosenu_server_create(budget_bytes, max_running=0, round_steps=0):
    lib = load()
    srv = lib.cosenu_server_create(int(budget_bytes), int(max_running), int(round_steps))
    if not srv:
        raise CosenuError(COSENU_EINVAL, lib.cosenu_server_last_error(None).decode())
    return srv


def cosenu_server_destroy(srv):
    load().cosenu_server_destroy(srv)


def cosenu_submit(srv, req):
    t = ctypes.c_uint64(0)
    _scheck(srv, load().cosenu_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return int(t.value)


def _result(r):
    c = r.conserved
    return {"status": r.status, "steps": r.steps, "t_submit": r.t_submit, "t_admit": r.t_admit,
            "t_done": r.t_done,
            "conserved": {"tr_nu": c.tr_nu, "tr_nubar": c.tr_nubar, "M": np.array(c.M[:]),
                          "M_vac": c.M_vac, "dP_max": c.dP_max, "dP_mean": c.dP_mean}}


def cosenu_poll(srv, ticket):
    """(rc, result dict): rc COSENU_PENDING while the run is unfinished, 0 once done."""
    r = cosenu_result()
    rc = _scheck(srv, load().cosenu_poll(srv, int(ticket), ctypes.byref(r)))
    return rc, _result(r)


def cosenu_wait(srv, ticket, timeout_s=-1.0):
    r = cosenu_result()
    rc = _scheck(srv, load().cosenu_wait(srv, int(ticket), float(timeout_s), ctypes.byref(r)))
    return rc, _result(r)


def cosenu_cancel(srv, ticket):
    return _scheck(srv, load().cosenu_cancel(srv, int(ticket)))


def cosenu_server_get_stats(srv):
    st = cosenu_server_stats()
    _scheck(srv, load().cosenu_server_get_stats(srv, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in cosenu_server_stats._fields_}


def cosenu_server_last_error(srv=None):
    return load().cosenu_server_last_error(srv).decode()


def make_request(nz, nv, L, scheme=COSENU_FDKO, precision=COSENU_MIXED, nsteps=1, state=None,
                 out_state=None, alpha=0.9, sigma_nu=0.6, sigma_nubar=0.5, eps0=1e-6, seed=12866,
                 **params):
    """A cosenu_request.  `state` / `out_state`: C-contiguous float64 numpy arrays (kept
    referenced by the returned object) or None.  Parameters not given take the library
    defaults (dt: 0.4 dz)."""
    p = cosenu_params(mu=1.0, omega=0.0, theta=0.0, lambda_=0.0, ko_eps=0.1, weno_eps=1e-6,
                      dt=0.0)
    for k, v in params.items():
        setattr(p, "lambda_" if k in ("lambda", "lam") else k, float(v))
    r = cosenu_request(nz=int(nz), nv=int(nv), L=float(L), scheme=int(scheme),
                       precision=int(precision), params=p, nsteps=int(nsteps),
                       state=None, alpha=float(alpha), sigma_nu=float(sigma_nu),
                       sigma_nubar=float(sigma_nubar), eps0=float(eps0), seed=int(seed),
                       out_state=None)
    for name, arr in (("state", state), ("out_state", out_state)):
        if arr is not None:
            assert arr.dtype == np.float64 and arr.flags["C_CONTIGUOUS"]
            assert arr.size == 8 * int(nz) * int(nv)
            setattr(r, name, _dptr(arr))
    r._keep = (state, out_state)
    return r


# ---------------------------------------------------------------- owner objects

class Solver:
    """Owns one handle: Solver(nz, nv, L, scheme, precision, **params)."""

    def __init__(self, nz, nv, L, scheme=COSENU_FDKO, precision=COSENU_FP64, **params):
        self.nz, self.nv, self.L = int(nz), int(nv), float(L)
        self.h = cosenu_create(nz, nv, L, scheme, precision)
        if params:
            cosenu_set_params(self.h, **params)

    def close(self):
        if self.h:
            cosenu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, host):
        cosenu_set_state(self.h, host)

    def state(self):
        out = np.empty((2, 4, self.nz, self.nv))
        cosenu_get_state(self.h, out)
        return out

    def rows(self, z0, nrows):
        out = np.empty((2, 4, nrows, self.nv))
        cosenu_get_rows(self.h, z0, nrows, out)
        return out

    def step(self, n=1):
        cosenu_step(self.h, n)

    def sync(self):
        cosenu_sync(self.h)

    def moments(self):
        zavg = np.empty((2, 4, self.nv))
        vmom = np.empty((self.nz, 6))
        cosenu_moments(self.h, zavg, vmom)
        return zavg, vmom

    def running_moments(self):
        return cosenu_running_moments(self.h, self.nz)

    def conserved(self):
        return cosenu_conserved(self.h)

    @property
    def params(self):
        p = cosenu_get_params(self.h)
        return {"mu": p.mu, "omega": p.omega, "theta": p.theta, "lambda": p.lambda_,
                "ko_eps": p.ko_eps, "weno_eps": p.weno_eps, "dt": p.dt}


class Member(Solver):
    """A grid of a Batch: the Solver calls, without ownership of the handle."""

    def __init__(self, batch, h, nz, nv, L):
        self.batch = batch
        self.nz, self.nv, self.L = int(nz), int(nv), float(L)
        self.h = h

    def close(self):
        self.h = None  # the batch owns the handle


class Batch:
    """Owns one batched solver; add() returns Member objects."""

    def __init__(self):
        self.b = cosenu_batch_create()
        self.members = []

    def close(self):
        if self.b:
            for m in self.members:
                m.h = None
            cosenu_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, nz, nv, L, scheme=COSENU_FDKO, precision=COSENU_MIXED, **params):
        h = cosenu_batch_add(self.b, nz, nv, L, scheme, precision)
        m = Member(self, h, nz, nv, L)
        if params:
            cosenu_set_params(h, **params)
        self.members.append(m)
        return m

    def remove(self, m):
        cosenu_batch_remove(self.b, m.h)
        self.members.remove(m)
        m.h = None

    def step(self, n=1):
        cosenu_batch_step(self.b, n)

    def sync(self):
        return cosenu_batch_sync(self.b)

    def tune(self, reps=2):
        return cosenu_batch_tune(self.b, reps)

    def classes(self):
        return [cosenu_batch_class_info(self.b, c) for c in range(cosenu_batch_classes(self.b))]

    def device_bytes(self):
        return cosenu_batch_device_bytes(self.b)


class Server:
    """Owns one serving loop: Server(budget_bytes, max_running=0, round_steps=0)."""

    def __init__(self, budget_bytes, max_running=0, round_steps=0):
        self.s = cosenu_server_create(budget_bytes, max_running, round_steps)
        self._reqs = {}

    def close(self):
        if self.s:
            cosenu_server_destroy(self.s)
            self.s = None
            self._reqs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, req):
        t = cosenu_submit(self.s, req)
        self._reqs[t] = req  # keeps the request's buffers alive until collected
        return t

    def poll(self, ticket):
        rc, res = cosenu_poll(self.s, ticket)
        if rc == COSENU_OK:
            self._reqs.pop(ticket, None)
        return rc, res

    def wait(self, ticket, timeout_s=-1.0):
        rc, res = cosenu_wait(self.s, ticket, timeout_s)
        if rc == COSENU_OK:
            self._reqs.pop(ticket, None)
        return rc, res

    def cancel(self, ticket):
        cosenu_cancel(self.s, ticket)

    def stats(self):
        return cosenu_server_get_stats(self.s)
