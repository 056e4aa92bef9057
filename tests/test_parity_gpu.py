"""GPU parity: the CUDA stage kernels against the FP64 oracle, element by element
on the same seeded inputs.

Tolerances.  FP64 path: max |delta rho| <= 1e-12 while the run stays in the
linear regime (|rho_ex| < 1e-3), the bound of the method's FP64 statement;
outside it (short nonlinear runs) the same bound over a few steps.  Mixed path:
relative error <= 1e-5 per component against the FP64 oracle in the linear
regime.
"""
import math

import numpy as np
import pytest

from paper_2203_12866_gb300 import binding, inputs
from parity_util import PRECS, SCHEMES, max_abs, rel_by_component, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_REL_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built(oracle):
    from paper_2203_12866_gb300 import build
    build.build()
    binding.load()


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
def test_fp64_collective_linear(scheme):
    nz, nv = 96, 32
    L = nz * (100.0 / 512)
    u0 = inputs.collective_state(nz, nv)
    got = run_gpu(u0, L, SCHEMES[scheme], PRECS["fp64"], 40, mu=1.0)
    ref = run_oracle(u0, L, SCHEMES[scheme], 40, mu=1.0)
    assert np.max(np.abs(ref[:, 2:])) < 1e-3
    assert max_abs(got, ref) <= FP64_TOL


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
def test_fp64_nonlinear_all_terms(scheme):
    """O(1) off-diagonals, vacuum term, matter term and nu-nu term all active."""
    nz, nv = 48, 16
    u0 = inputs.random_state(nz, nv, seed=31, offdiag=0.3)
    kw = dict(mu=1.3, omega=0.4, theta=0.25, ko_eps=0.1)
    kw["lambda"] = 0.2
    got = run_gpu(u0, 7.0, SCHEMES[scheme], PRECS["fp64"], 6, **kw)
    ref = run_oracle(u0, 7.0, SCHEMES[scheme], 6, **kw)
    assert max_abs(got, ref) <= FP64_TOL


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
@pytest.mark.parametrize("nz,nv", [(37, 36), (53, 12), (200, 100)])
def test_fp64_ragged_tiles(scheme, nz, nv):
    """z ranges that do not divide into the CTAs evenly, v not a multiple of 32."""
    u0 = inputs.random_state(nz, nv, seed=nz + nv, offdiag=0.05)
    got = run_gpu(u0, 0.2 * nz, SCHEMES[scheme], PRECS["fp64"], 3, mu=0.7, omega=0.2, theta=0.3)
    ref = run_oracle(u0, 0.2 * nz, SCHEMES[scheme], 3, mu=0.7, omega=0.2, theta=0.3)
    assert max_abs(got, ref) <= FP64_TOL


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
@pytest.mark.parametrize("nz,nv", [(37, 36), (53, 12), (200, 100), (61, 4)])
def test_mixed_ragged_tiles(scheme, nz, nv):
    """Mixed path on ragged shapes: odd row counts per CTA (the two-row march of
    mixed WENO7 ends on a single row), and v-row lengths whose increment-kernel
    chunks hold a non-power-of-two number of plane-rows (nv = 36: 113 rows of 9
    groups; nv = 12: 341 of 3; nv = 100: 40 of 25; nv = 4: 1024 of 1)."""
    u0 = inputs.random_state(nz, nv, seed=nz + nv, offdiag=0.05)
    got = run_gpu(u0, 0.2 * nz, SCHEMES[scheme], PRECS["mixed"], 6, mu=0.7, omega=0.2, theta=0.3)
    ref = run_oracle(u0, 0.2 * nz, SCHEMES[scheme], 6, mu=0.7, omega=0.2, theta=0.3)
    assert rel_by_component(got, ref) <= MIXED_REL_TOL


@pytest.mark.parametrize("scheme", ["fdko", "weno7"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nz,nv", [(600, 252), (911, 132), (1000, 256)])
def test_wide_rows(scheme, prec, nz, nv):
    """Long v-rows with several rows per CTA: nv = 252 and 256 give the mixed
    WENO7 kernel 16 consumer warps and three reducer warps taking the rows in
    turn (nv = 252 and 132 leave the reducers' second column chunk partly
    empty); nv = 252 and 132 put both species in one warp (the consumers apply
    the moments' species sign), nv = 256 one species per warp (the reducer
    applies it per warp)."""
    u0 = inputs.random_state(nz, nv, seed=nz + nv, offdiag=0.05)
    kw = dict(mu=0.7, omega=0.2, theta=0.3)
    got = run_gpu(u0, 0.2 * nz, SCHEMES[scheme], PRECS[prec], 6, **kw)
    ref = run_oracle(u0, 0.2 * nz, SCHEMES[scheme], 6, **kw)
    if prec == "fp64":
        assert max_abs(got, ref) <= FP64_TOL
    else:
        assert rel_by_component(got, ref) <= MIXED_REL_TOL


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nz", [1, 2, 3, 5, 9])
def test_tiny_periodic_grids(scheme, prec, nz):
    """Grids shorter than the stencil: the halo wraps around the period several times."""
    nv = 8
    u0 = inputs.random_state(nz, nv, seed=100 + nz, offdiag=0.05)
    got = run_gpu(u0, 0.3 * nz, SCHEMES[scheme], PRECS[prec], 4, mu=1.0, omega=0.1, theta=0.2)
    ref = run_oracle(u0, 0.3 * nz, SCHEMES[scheme], 4, mu=1.0, omega=0.1, theta=0.2)
    if prec == "fp64":
        assert max_abs(got, ref) <= FP64_TOL
    else:
        assert rel_by_component(got, ref) <= MIXED_REL_TOL


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
def test_mixed_collective_linear(scheme):
    nz, nv = 160, 64
    L = nz * (100.0 / 512)
    u0 = inputs.collective_state(nz, nv)
    got = run_gpu(u0, L, SCHEMES[scheme], PRECS["mixed"], 60, mu=1.0)
    ref = run_oracle(u0, L, SCHEMES[scheme], 60, mu=1.0)
    assert np.max(np.abs(ref[:, 2:])) < 1e-3
    assert rel_by_component(got, ref) <= MIXED_REL_TOL


def test_config_small_full_run():
    """nz = 512, nv = 32, z in [-50, 50), dt = 0.4 dz, 400 FD+KO FP64 steps, mu = 1,
    alpha = 0.9, sigma = (0.6, 0.5), random-phase seed 1e-6 -- the whole run."""
    nz, nv, L = 512, 32, 100.0
    u0 = inputs.collective_state(nz, nv, alpha=0.9, sigma_nu=0.6, sigma_nubar=0.5, eps0=1e-6)
    got = run_gpu(u0, L, SCHEMES["fdko"], PRECS["fp64"], 400, mu=1.0)
    ref = run_oracle(u0, L, SCHEMES["fdko"], 400, mu=1.0)
    assert np.max(np.abs(ref[:, 2:])) < 1e-3
    assert max_abs(got, ref) <= FP64_TOL


def test_graph_replay_equals_single_steps():
    nz, nv = 64, 16
    u0 = inputs.random_state(nz, nv, seed=5, offdiag=0.1)
    with binding.Solver(nz, nv, 10.0, 0, 0, mu=1.0, omega=0.2, theta=0.1) as s:
        s.set_state(u0)
        s.step(7)  # graph of 2 steps x 3 + one direct step
        a = s.state()
        s.set_state(u0)
        for _ in range(7):
            s.step(1)
        b = s.state()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_deterministic(prec):
    nz, nv = 300, 64
    u0 = inputs.collective_state(nz, nv)
    a = run_gpu(u0, 60.0, 1, PRECS[prec], 5)
    b = run_gpu(u0, 60.0, 1, PRECS[prec], 5)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("scheme", ["fdko", "weno7", "fdko3"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_conservation_on_gpu(scheme, prec, oracle):
    nz, nv = 128, 32
    u0 = inputs.random_state(nz, nv, seed=77, offdiag=0.2)
    with binding.Solver(nz, nv, 20.0, SCHEMES[scheme], PRECS[prec], mu=1.0) as s:
        s.set_state(u0)
        c0 = s.conserved()
        s.step(20)
        s.sync()
        c1 = s.conserved()
    tol = 1e-13 if prec == "fp64" else 1e-7
    assert abs(c1["tr_nu"] - c0["tr_nu"]) <= tol * abs(c0["tr_nu"])
    assert abs(c1["tr_nubar"] - c0["tr_nubar"]) <= tol * abs(c0["tr_nubar"])
    assert np.max(np.abs(c1["M"] - c0["M"])) <= tol * np.max(np.abs(c0["M"]))
    assert c1["step"] == 20


def test_diagnostics_match_oracle(oracle):
    nz, nv = 70, 24
    u0 = inputs.random_state(nz, nv, seed=3, offdiag=0.3)
    with binding.Solver(nz, nv, 9.0, 0, 0, theta=0.4) as s:
        s.set_state(u0)
        zavg, vmom = s.moments()
        c = s.conserved()
        rows = s.rows(10, 7)
    p = oracle.params(nz, nv, 9.0, theta=0.4)
    oz, om = oracle.moments(p, u0)
    oc = oracle.conserved(p, u0)
    assert np.max(np.abs(zavg - oz)) < 1e-14
    assert np.max(np.abs(vmom - om)) < 1e-14
    for k in ("tr_nu", "tr_nubar", "M_vac", "dP_max", "dP_mean"):
        assert c[k] == pytest.approx(oc[k], rel=1e-12, abs=1e-15), k
    assert np.allclose(c["M"], oc["M"], rtol=1e-12, atol=1e-15)
    assert np.array_equal(rows, u0[:, :, 10:17])


def test_nonfinite_is_reported():
    nz, nv = 32, 8
    u0 = inputs.random_state(nz, nv, seed=1)
    u0[0, 2, 5, 3] = np.nan
    with binding.Solver(nz, nv, 5.0, 0, 0) as s:
        s.set_state(u0)
        s.step(1)
        with pytest.raises(binding.CosenuError) as e:
            s.sync()
        assert e.value.code == binding.COSENU_ENONFINITE
        s.sync()  # the flag is cleared once reported


def test_bad_state_length_rejected():
    with binding.Solver(16, 8, 1.0) as s:
        with pytest.raises(binding.CosenuError) as e:
            s.set_state(np.zeros(10))
        assert e.value.code == binding.COSENU_EINVAL


def test_vacuum_homogeneous_exact_map():
    """mu = 0, omega = 0.5, theta = 0.1, z-uniform pure nu_e: every cell follows the
    RK4 map of the Bloch precession, on a grid that spans many CTAs."""
    nz, nv, L = 4096, 128, 3200.0 * 4096 / 65536
    u0 = np.zeros((2, 4, nz, nv))
    u0[:, 0] = 1.0
    n = 50
    for prec, tol in (("fp64", 1e-13), ("mixed", 2e-6)):
        with binding.Solver(nz, nv, L, 0, PRECS[prec], mu=0.0, omega=0.5, theta=0.1) as s:
            s.set_state(u0)
            dt = s.params["dt"]
            s.step(n)
            got = s.state()
        B = np.array([math.sin(0.2), 0.0, -math.cos(0.2)])
        A = 0.5 * np.array([[0, -B[2], B[1]], [B[2], 0, -B[0]], [-B[1], B[0], 0]])
        Z = dt * A
        M = np.linalg.matrix_power(np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24, n)
        P = M @ np.array([0.0, 0.0, 1.0])
        exp = np.array([(1 + P[2]) / 2, (1 - P[2]) / 2, P[0] / 2, -P[1] / 2])
        assert np.max(np.abs(got - exp[None, :, None, None])) <= tol, prec
