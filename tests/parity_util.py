"""Shared helpers of the GPU parity tests: run the same seeded input through the
CUDA library (via the C ABI binding) and through the oracle."""
import numpy as np

import oracle
from paper_2203_12866_gb300 import binding

SCHEMES = {"fdko": binding.COSENU_FDKO, "weno7": binding.COSENU_WENO7,
           "fdko3": binding.COSENU_FDKO3}
PRECS = {"fp64": binding.COSENU_FP64, "mixed": binding.COSENU_MIXED}


def run_gpu(u0, L, scheme, prec, nsteps, **params):
    nz, nv = u0.shape[2], u0.shape[3]
    with binding.Solver(nz, nv, L, scheme, prec, **params) as s:
        s.set_state(u0)
        s.step(nsteps)
        s.sync()
        return s.state()


def run_oracle(u0, L, scheme, nsteps, **params):
    nz, nv = u0.shape[2], u0.shape[3]
    kw = dict(params)
    if "lambda" in kw:
        kw["lam"] = kw.pop("lambda")
    p = oracle.params(nz, nv, L, scheme, **kw)
    return oracle.step(p, u0, nsteps)


def max_abs(a, b):
    return float(np.max(np.abs(a - b)))


def rel_by_component(got, ref):
    """max over (species, component) of max|got - ref| / max|ref| of that component."""
    worst = 0.0
    for s in range(2):
        for c in range(4):
            scale = float(np.max(np.abs(ref[s, c])))
            if scale == 0.0:
                continue
            worst = max(worst, float(np.max(np.abs(got[s, c] - ref[s, c]))) / scale)
    return worst
