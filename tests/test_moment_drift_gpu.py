"""Mixed precision: the running FP64 v-moments D_n(y) from which the stage kernels
form H_nunu, against the moments recomputed from y in double.

The mixed path does not re-sum the v-moments of the state every stage.  It keeps
D_n(y) = sum_j w_j v_j^n (S_j - Sbar_j^*) (Eq. (ham)) as a per-z double running
sum: set from y when the state is replaced, then advanced every RK4 step by the
v-sums of the step's increment dy (the same float dy that is added to y exactly,
float to double).  The increment kernel forms those v-sums as float pairs
(hi + lo) with the products' and additions' rounding errors recovered exactly
and the double weights w_j, w_j v_j split into float pairs, so the running sums
follow D_n(y) to double precision: what remains is the double rounding of
y + dy, at most 2^-53 |y| per element and step.  The bound checked is therefore
(steps + 64) 2^-52 times the moment's magnitude sum_j w_j |v_j|^n (|terms|) (the
64 covering the double summation of D_n(y) itself); a running sum advanced by
plain float v-sums misses it by five to six orders of magnitude (measured: 1e-7
to 6e-7 of the moments after 4000-6400 steps).

Workloads: the medium one, 65536 x 128 on [-1600, 1600), mu = 1, alpha = 0.9
and 1.0, FD4+KO and WENO7, 4000 steps (linear regime); the first one, 512 x 32
on [-50, 50), mu = 1, run to t = 500, past the saturation of the fast
instability (6400 steps).
"""
import numpy as np
import pytest

from paper_2203_12866_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

NAMES = ("D3_0", "D3_1", "Dr_0", "Dr_1", "Di_0", "Di_1")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2203_12866_gb300 import build
    build.build()
    binding.load()


def _magnitudes(y, nv):
    """max over z of sum_j w_j |v_j|^n times the absolute terms of each moment."""
    v = -1.0 + (np.arange(nv) + 0.5) * (2.0 / nv)
    w = np.full(nv, 2.0 / nv)
    terms = (np.abs(y[0, 0] - y[0, 1]) + np.abs(y[1, 0] - y[1, 1]),
             np.abs(y[0, 2]) + np.abs(y[1, 2]), np.abs(y[0, 3]) + np.abs(y[1, 3]))
    out = []
    for t in terms:
        for n in (0, 1):
            out.append(float(np.max(t @ (w * np.abs(v) ** n))))
    return out


def _drift(s):
    run = s.running_moments()
    _, ref = s.moments()
    mags = _magnitudes(s.state(), s.nv)
    return {name: (float(np.max(np.abs(run[:, k] - ref[:, k]))), mags[k])
            for k, name in enumerate(NAMES)}


def _check(label, s, nsteps):
    d = _drift(s)
    print(label + ": " + ", ".join(f"{n} {e:.2e} of magnitude {m:.2e}" for n, (e, m) in d.items()))
    tol = (nsteps + 64) * 2.0 ** -52
    for n, (e, m) in d.items():
        assert e <= tol * m, (label, n, e, m, tol)


@pytest.mark.parametrize("scheme,alpha", [(binding.COSENU_FDKO, 0.9), (binding.COSENU_FDKO, 1.0),
                                          (binding.COSENU_WENO7, 0.9)])
def test_running_moments_medium_workload(scheme, alpha):
    nz, nv, L = 65536, 128, 3200.0
    u0 = inputs.collective_state(nz, nv, alpha=alpha)
    with binding.Solver(nz, nv, L, scheme, binding.COSENU_MIXED, mu=1.0) as s:
        s.set_state(u0)
        before = _drift(s)
        assert all(e == 0.0 for e, _ in before.values())  # set from y by the same sums
        s.step(4000)
        s.sync()
        _check(f"65536x128 scheme {scheme} alpha {alpha}, 4000 steps", s, 4000)


@pytest.mark.parametrize("scheme", [binding.COSENU_FDKO, binding.COSENU_WENO7])
def test_running_moments_after_saturation(scheme):
    nz, nv, L = 512, 32, 100.0
    u0 = inputs.collective_state(nz, nv)
    with binding.Solver(nz, nv, L, scheme, binding.COSENU_MIXED, mu=1.0) as s:
        s.set_state(u0)
        n = int(round(500.0 / s.params["dt"]))
        s.step(n)
        s.sync()
        assert np.max(np.abs(s.state()[:, 2:])) > 0.3  # saturated
        _check(f"512x32 scheme {scheme}, {n} steps to t = 500", s, n)
