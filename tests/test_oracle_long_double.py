"""Whole-step pin of the oracle's rounding: the FP64 oracle against a copy of the
same C source in which every double (and every floating literal) is long double.

On tiny grids (nz = 16, nv = 4 and 8) with every term active -- advection of each
scheme, Kreiss-Oliger, vacuum, matter and nu-nu terms, O(1) off-diagonals -- a
few RK4 steps computed in double must agree with the extended-precision run to a
small multiple of the double rounding.  A formula in the oracle that loses
accuracy to cancellation or to a badly conditioned order of operations would
show up as a larger difference.  (The copy is made textually at test time; the
product never sees it.)"""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2203_12866_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(oracle.__file__))


def _long_double_copy(src_text):
    # floating literals first (1.0, 2.5e-3, .5): add the long double suffix
    txt = re.sub(r"(?<![\w.])((?:\d+\.\d*|\.\d+)(?:[eE][+-]?\d+)?)(?![\w.])", r"\1L", src_text)
    txt = re.sub(r"(?<!long )\bdouble\b", "long double", txt)
    return txt


class LDParams(ctypes.Structure):
    LD = ctypes.c_longdouble
    _fields_ = [("nz", ctypes.c_int64), ("nv", ctypes.c_int32), ("L", LD),
                ("scheme", ctypes.c_int32), ("hmode", ctypes.c_int32), ("mu", LD),
                ("omega", LD), ("theta", LD), ("lam", LD), ("ko_eps", LD), ("weno_eps", LD),
                ("dt", LD), ("vgrid", ctypes.c_int32)]


@pytest.fixture(scope="module")
def ld_lib(tmp_path_factory):
    cc = shutil.which("gcc")
    if cc is None or ctypes.sizeof(ctypes.c_longdouble) <= 8:
        pytest.skip("needs gcc and a long double wider than double")
    d = tmp_path_factory.mktemp("oracle_ld")
    src = open(os.path.join(HERE, "cosenu_oracle.c")).read()
    hdr = open(os.path.join(HERE, "cosenu_oracle.h")).read()
    src = src.replace("#include <math.h>", "#include <tgmath.h>")
    assert "#include <tgmath.h>" in src
    (d / "cosenu_oracle.c").write_text(_long_double_copy(src))
    (d / "cosenu_oracle.h").write_text(_long_double_copy(hdr))
    so = d / "libld.so"
    subprocess.run([cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    f"-I{d}", "-o", str(so), str(d / "cosenu_oracle.c"), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_step.argtypes = [ctypes.POINTER(LDParams), ctypes.c_void_p, ctypes.c_int64]
    return lib


def _ld_step(lib, p, u, n):
    q = LDParams(p.nz, p.nv, p.L, p.scheme, p.hmode, p.mu, p.omega, p.theta, p.lam, p.ko_eps,
                 p.weno_eps, p.dt, p.vgrid)
    y = np.ascontiguousarray(u, dtype=np.longdouble).copy()
    assert lib.oracle_step(ctypes.byref(q), y.ctypes.data, int(n)) == 0
    return y


def test_copy_is_really_extended(ld_lib):
    """The copy computes in extended precision: a case whose double result carries
    rounding differs from it in the last bits (guards against a copy that silently
    kept double arithmetic)."""
    p = oracle.params(16, 4, 3.3, oracle.FDKO, mu=1.1, omega=0.3, theta=0.2)
    u0 = inputs.random_state(16, 4, seed=11, offdiag=0.4)
    a = oracle.step(p, u0, 3)
    b = _ld_step(ld_lib, p, u0, 3)
    assert np.max(np.abs(a - b.astype(np.float64))) > 0.0


# Allowed difference relative to max |u|.  FD4+KO: a few roundings of the stencil
# sums.  WENO7: the printed smoothness indicators (Eq. (Si4)) are quadratic forms
# with coefficients up to 1.7e4 whose terms largely cancel, so their double
# rounding reaches the weights amplified by about 1e1 (measured 4-5e-15).
TOL = {oracle.FDKO: 2e-15, oracle.FDKO3: 2e-15, oracle.WENO7: 2e-14}


@pytest.mark.parametrize("scheme", [oracle.FDKO, oracle.WENO7, oracle.FDKO3])
@pytest.mark.parametrize("nv", [4, 8])
def test_whole_steps_match_long_double_copy(ld_lib, scheme, nv):
    nz = 16
    p = oracle.params(nz, nv, 0.37 * nz, scheme, mu=1.3, omega=0.4, theta=0.25, lam=0.2)
    u0 = inputs.random_state(nz, nv, seed=40 + nv + scheme, offdiag=0.3)
    a = oracle.step(p, u0, 5)
    b = _ld_step(ld_lib, p, u0, 5)
    err = float(np.max(np.abs(a - b.astype(np.float64))))
    assert err <= TOL[scheme] * float(np.max(np.abs(u0))), err
