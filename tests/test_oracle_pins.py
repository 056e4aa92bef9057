"""Pins of the FP64 oracle against what arXiv:2203.12866 and the mathematics fix.

Nothing here compares the oracle with itself or with the CUDA path.  Each test
uses an independent route to the same result: Fourier symbols derived from the
operator definitions, exact polynomial cell averages, the textbook RK4
stability polynomial, the closed-form vacuum solution, discrete conservation
laws, and the linear dispersion relation solved with numpy.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2203_12866_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rk4_poly(z):
    """Stability polynomial of classical RK4 (exact for linear autonomous systems)."""
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def central_difference_weights(offsets, order=1):
    """Weights c_m with sum c_m f(x + m h) = h^order f^(order)(x) + O(h^len), from
    the Taylor moment conditions (no tabulated coefficients)."""
    n = len(offsets)
    A = np.array([[m ** q for m in offsets] for q in range(n)], dtype=float)
    b = np.zeros(n)
    b[order] = math.factorial(order)
    return np.linalg.solve(A, b)


def fd4_ko_symbol(theta, h, v, eps, r=2):
    """Fourier symbol of -v d/dz (4th-order central) - Q, with
    Q = eps (-1)^r h^(2r-1) (D+)^r (D-)^r / 2^(2r) applied on the time-derivative side."""
    offs = [-2, -1, 0, 1, 2]
    c = central_difference_weights(offs)
    ddz = sum(cm * np.exp(1j * m * theta) for m, cm in zip(offs, c)) / h
    dplus = (np.exp(1j * theta) - 1.0) / h
    dminus = (1.0 - np.exp(-1j * theta)) / h
    Q = eps * (-1) ** r * h ** (2 * r - 1) * dplus ** r * dminus ** r / 2 ** (2 * r)
    return -v * ddz - Q


def advect_dft(u, lam_of_theta, dt, nsteps):
    """Exact discrete solution of du/dt = L u (L circulant in z) under RK4."""
    nz = u.shape[-2]
    theta = 2 * np.pi * np.fft.fftfreq(nz)
    uh = np.fft.fft(u, axis=-2)
    out = np.empty_like(u)
    for j in range(u.shape[-1]):
        lam = lam_of_theta(theta, j)
        out[..., :, j] = np.real(np.fft.ifft(uh[..., :, j] * rk4_poly(dt * lam) ** nsteps, axis=-1))
    return out


# --------------------------------------------------------------------------- grid


def test_vgrid_midpoints(oracle):
    g = GOLDEN["beam_v_nv100"]
    v, w = oracle.vgrid(g["nv"])
    assert v[-1] == pytest.approx(g["v"], abs=1e-15)
    assert np.allclose(w, 2.0 / g["nv"])
    assert v[0] == pytest.approx(-g["v"], abs=1e-15)
    assert np.all(np.diff(v) > 0)


@pytest.mark.parametrize("nv", [4, 8, 12, 9, 33])
def test_vgrid_vertex_quadratures(oracle, nv):
    """Sec. 3.1 vertex grids: v_j = -1 + j h on [-1, 1].  The trapezoid rule
    integrates polynomials of degree <= 1 exactly and v^2 with the composite
    error h^2 / 3; Simpson's rule (with a 3/8 panel closing an odd interval
    count) integrates degree <= 3 exactly; all weights are positive."""
    exact = [2.0, 0.0, 2.0 / 3.0, 0.0, 2.0 / 5.0]
    h = 2.0 / (nv - 1)
    v, w = oracle.vgrid(nv, oracle.TRAPEZOID)
    assert v[0] == -1.0 and v[-1] == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.diff(v), h, atol=1e-15) and np.all(w > 0)
    for k in (0, 1):
        assert np.sum(w * v ** k) == pytest.approx(exact[k], abs=1e-14)
    assert np.sum(w * v ** 2) == pytest.approx(2.0 / 3.0 + h * h / 3.0, abs=1e-14)
    v, w = oracle.vgrid(nv, oracle.SIMPSON)
    assert np.all(w > 0)
    for k in range(4):
        assert np.sum(w * v ** k) == pytest.approx(exact[k], abs=1e-14)
    if (nv - 1) % 2 == 0:  # pure 1/3 rule: error of v^4 is -4 h^4 / 15
        assert np.sum(w * v ** 4) == pytest.approx(exact[4] + 4.0 * h ** 4 / 15.0, abs=1e-14)
    else:  # the 3/8 panel makes the rule no longer exact for v^4
        assert abs(np.sum(w * v ** 4) - exact[4]) > 1e-8


@pytest.mark.parametrize("mode", [1, 2])
def test_moments_vertex_quadratures_exact_for_linear_profiles(oracle, mode):
    """With S_ee - S_xx = 1 + v, D3_0 = int (1 + v) dv = 2 and D3_1 = int (v + v^2) dv
    = 2/3 (Simpson, exact to degree 3) or 2/3 + h^2/3 (trapezoid)."""
    nz, nv = 4, 12
    v, _ = oracle.vgrid(nv, mode)
    u = np.zeros((2, 4, nz, nv))
    u[0, 0] = (1 + v)[None, :]
    _, vmom = oracle.moments(oracle.params(nz, nv, 1.0, vgrid=mode), u)
    h = 2.0 / (nv - 1)
    assert np.allclose(vmom[:, 0], 2.0, atol=1e-14)
    d31 = 2.0 / 3.0 + (h * h / 3.0 if mode == 1 else 0.0)
    assert np.allclose(vmom[:, 1], d31, atol=1e-14)


# --------------------------------------------------------------------------- WENO7


def f4_golden():
    g = GOLDEN["weno7_f4"]
    return [g[f"S{r}"] for r in range(4)]


def test_weno7_constant_data(oracle):
    val, det = oracle.weno7_face(np.full(7, 2.5), 1e-6, detail=True)
    assert val == pytest.approx(2.5, rel=1e-15)
    assert np.all(det["si"] == 0.0)
    assert np.allclose(det["f4"], 2.5, rtol=1e-15)


def cell_averages(coef, offsets):
    """Exact cell averages over [m - 1/2, m + 1/2] (h = 1) of the polynomial sum coef[k] x^k."""
    P = np.polynomial.polynomial
    I = P.polyint(coef)
    return np.array([P.polyval(m + 0.5, I) - P.polyval(m - 0.5, I) for m in offsets])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_weno7_cubic_reconstructed_exactly(oracle, seed):
    """Every 4-cell sub-stencil reproduces a cubic exactly, so the WENO value at
    i+1/2 is exact whatever the nonlinear weights are (Eq. (f4s), (fn_w_lin_comb))."""
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal(4)
    f = cell_averages(coef, range(-3, 4))
    exact = np.polynomial.polynomial.polyval(0.5, coef)
    val, det = oracle.weno7_face(f, 1e-6, detail=True)
    assert np.allclose(det["f4"], exact, atol=1e-13)
    assert val == pytest.approx(exact, abs=1e-13)
    # the printed sub-stencil coefficients give the same four numbers
    for r, S in enumerate(f4_golden()):
        ref = sum(n * f[o + 3] for o, n in zip(S["offsets"], S["num"])) / 12.0
        assert det["f4"][r] == pytest.approx(ref, abs=1e-14)


def test_weno7_linear_weights_reproduce_eq_f7(oracle):
    """With epsilon >> SI the weights are the linear ones and the result must be the
    7th-order value of Eq. (f7).  This fixes which d_r belongs to which sub-stencil."""
    c7 = np.array([n / d for n, d in GOLDEN["weno7_f7"]["coeffs"]])
    rng = np.random.default_rng(7)
    for _ in range(5):
        f = rng.standard_normal(7)
        val, det = oracle.weno7_face(f, 1e30, detail=True)
        assert val == pytest.approx(float(c7 @ f), abs=1e-13)
    d_printed = np.array(GOLDEN["weno7_d_printed"]["num_over_35"]) / 35.0
    # the weights used belong to S_0..S_3 in the reverse of the printed order
    assert np.allclose(det["wbar"], d_printed[::-1], atol=1e-15)
    # and a degree-6 polynomial is reconstructed exactly with those weights
    coef = rng.standard_normal(7)
    f = cell_averages(coef, range(-3, 4))
    assert oracle.weno7_face(f, 1e30) == pytest.approx(
        np.polynomial.polynomial.polyval(0.5, coef), abs=1e-12)


def jiang_shu_beta(vals, offsets):
    """Smoothness integral sum_{l=1..3} int_{-1/2}^{1/2} (p^(l))^2 dx (h = 1) of the cubic
    whose cell averages on `offsets` are `vals`."""
    P = np.polynomial.polynomial
    A = np.array([[((o + 0.5) ** (k + 1) - (o - 0.5) ** (k + 1)) / (k + 1) for k in range(4)]
                  for o in offsets])
    c = np.linalg.solve(A, vals)
    b = 0.0
    for l in range(1, 4):
        d = P.polyder(c, l)
        I = P.polyint(P.polymul(d, d))
        b += P.polyval(0.5, I) - P.polyval(-0.5, I)
    return b


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_weno7_smoothness_index_is_scaled_jiang_shu(oracle, seed):
    """The integer forms of Eq. (Si4) are 240 x the Jiang-Shu smoothness integral of
    each sub-stencil's cubic (independent polynomial computation)."""
    f = np.random.default_rng(seed).standard_normal(7)
    _, det = oracle.weno7_face(f, 1e-6, detail=True)
    for r, S in enumerate(f4_golden()):
        beta = jiang_shu_beta(f[np.array(S["offsets"]) + 3], S["offsets"])
        assert det["si"][r] == pytest.approx(240.0 * beta, rel=1e-12, abs=1e-12)


def test_weno7_weight_formula(oracle):
    """w_r = d_r / (SI_r + eps)^2, normalised (Eq. (weight)), for a rough stencil."""
    f = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 1.0])
    eps = 1e-6
    _, det = oracle.weno7_face(f, eps, detail=True)
    d = np.array(GOLDEN["weno7_d_printed"]["num_over_35"])[::-1] / 35.0
    w = d / (det["si"] + eps) ** 2
    assert np.allclose(det["wbar"], w / w.sum(), rtol=1e-14)
    # the only smooth sub-stencil is S_0 = {i..i+3} (all ones): it takes the weight
    assert det["wbar"][0] > 1 - 1e-9


# --------------------------------------------------------------------------- advection


@pytest.mark.parametrize("ko_eps", [0.0, 0.1])
def test_fdko_pure_advection_equals_dft_solution(oracle, ko_eps):
    """mu = omega = 0: the scheme is linear and circulant, so each Fourier mode is
    multiplied per step by the RK4 polynomial of dt x (symbol of the operator)."""
    nz, nv, L = 32, 4, 11.0
    p = oracle.params(nz, nv, L, oracle.FDKO, mu=0.0, ko_eps=ko_eps, cfl=0.4)
    u0 = inputs.random_state(nz, nv, seed=5, offdiag=1.0)
    got = oracle.step(p, u0, 25)
    v, _ = oracle.vgrid(nv)
    h = L / nz
    ref = advect_dft(u0, lambda th, j: fd4_ko_symbol(th, h, v[j], ko_eps), p.dt, 25)
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("ko_eps", [0.1, 0.7])
def test_fdko3_pure_advection_equals_dft_solution(oracle, ko_eps):
    """Kreiss-Oliger with r = 3 (the general Q of Sec. 3.1 at r = 3): same exact
    discrete solution, with the r = 3 symbol built from D+ and D-."""
    nz, nv, L = 32, 4, 11.0
    p = oracle.params(nz, nv, L, oracle.FDKO3, mu=0.0, ko_eps=ko_eps, cfl=0.4)
    u0 = inputs.random_state(nz, nv, seed=15, offdiag=1.0)
    got = oracle.step(p, u0, 25)
    v, _ = oracle.vgrid(nv)
    h = L / nz
    ref = advect_dft(u0, lambda th, j: fd4_ko_symbol(th, h, v[j], ko_eps, r=3), p.dt, 25)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_ko3_is_dissipative_and_weaker_at_long_waves():
    """r = 3: -eps sin^6(theta/2) / h, dissipative; smaller than r = 2 for every
    theta < pi (sin^6 <= sin^4), equal at the grid scale."""
    theta = np.linspace(0, np.pi, 101)
    s3 = fd4_ko_symbol(theta, 0.5, 0.0, 0.1, r=3)
    s2 = fd4_ko_symbol(theta, 0.5, 0.0, 0.1, r=2)
    assert np.all(s3.real <= 1e-15)
    assert s3.real[-1] == pytest.approx(-0.1 / 0.5, rel=1e-12)
    assert np.all(s3.real >= s2.real - 1e-15)
    assert np.allclose(s3.real, -0.1 / 0.5 * np.sin(theta / 2) ** 6, atol=1e-15)


def test_ko_is_dissipative(oracle):
    """The Kreiss-Oliger term removes energy at every mode (reading of Sec. 3.1)."""
    theta = np.linspace(0, np.pi, 101)
    sym = fd4_ko_symbol(theta, 0.5, 0.0, 0.1)
    assert np.all(sym.real <= 1e-15)
    assert sym.real[-1] == pytest.approx(-0.1 / 0.5, rel=1e-12)


def weno7_linear_symbol(theta, h, v):
    """Linear-weight WENO7 (Eq. (f7)), upwind by the sign of v, in Fourier space:
    -(F_{i+1/2} - F_{i-1/2}) / h with F = v x reconstruction."""
    c7 = [n / d for n, d in GOLDEN["weno7_f7"]["coeffs"]]
    if v > 0:
        face = sum(c * np.exp(1j * m * theta) for m, c in zip(range(-3, 4), c7))
    else:
        face = sum(c * np.exp(1j * (1 - m) * theta) for m, c in zip(range(-3, 4), c7))
    return -v * face * (1.0 - np.exp(-1j * theta)) / h


def test_weno7_linear_limit_equals_dft_solution(oracle):
    nz, nv, L = 32, 4, 9.0
    p = oracle.params(nz, nv, L, oracle.WENO7, mu=0.0, weno_eps=1e30, cfl=0.4)
    u0 = inputs.random_state(nz, nv, seed=6, offdiag=1.0)
    got = oracle.step(p, u0, 20)
    v, _ = oracle.vgrid(nv)
    ref = advect_dft(u0, lambda th, j: weno7_linear_symbol(th, L / nz, v[j]), p.dt, 20)
    assert np.max(np.abs(got - ref)) < 1e-12


def gaussian_run(oracle, scheme, nz, t_end, dt, ko_eps=0.1, weno_eps=1e-6, cell_avg=False):
    """Advect a unit Gaussian (width 1) on z in [-10, 10) for time t_end at v = +-0.5."""
    from scipy.special import erf
    L, nv = 20.0, 2
    h = L / nz
    zc = -L / 2 + (np.arange(nz) + 0.5) * h
    def prof(z):
        if cell_avg:
            a, b = z - h / 2, z + h / 2
            return np.sqrt(np.pi / 2) * (erf(b / np.sqrt(2)) - erf(a / np.sqrt(2))) / h
        return np.exp(-z * z / 2)
    u0 = np.zeros((2, 4, nz, nv))
    u0[:, :, :, :] = prof(zc)[None, None, :, None]
    nsteps = int(round(t_end / dt))
    p = oracle.params(nz, nv, L, scheme, mu=0.0, ko_eps=ko_eps, weno_eps=weno_eps, dt=dt)
    u = oracle.step(p, u0, nsteps)
    v = np.array([-0.5, 0.5])
    err = []
    for j in range(nv):
        shift = v[j] * nsteps * dt
        zz = (zc - shift + L / 2) % L - L / 2
        err.append(np.sqrt(np.mean((u[0, 0, :, j] - prof(zz)) ** 2)))
    return max(err)


@pytest.mark.slow
def test_convergence_orders(oracle):
    """Observed orders with a time step small enough that RK4 error is negligible:
    FD4 without KO -> 4, FV WENO7 (linear weights) -> 7, FV WENO7 (eps = 1e-6) >= 5
    (Sec. 4.1, Fig. 2 discussion and Appendix C; KO lowers the FD order)."""
    dt = 2e-3
    e = [gaussian_run(oracle, oracle.FDKO, n, 1.0, dt, ko_eps=0.0) for n in (80, 160)]
    assert 3.8 < math.log2(e[0] / e[1]) < 4.2
    e = [gaussian_run(oracle, oracle.WENO7, n, 1.0, dt, weno_eps=1e30, cell_avg=True)
         for n in (80, 160)]
    assert 6.6 < math.log2(e[0] / e[1]) < 7.4
    e = [gaussian_run(oracle, oracle.WENO7, n, 1.0, dt, cell_avg=True) for n in (80, 160)]
    assert math.log2(e[0] / e[1]) > 5.5
    e = [gaussian_run(oracle, oracle.FDKO, n, 1.0, dt, ko_eps=0.1) for n in (80, 160)]
    assert 3.0 < math.log2(e[0] / e[1]) < 3.8
    # r = 3 dissipation is O(h^5): the FD4 order survives
    e = [gaussian_run(oracle, oracle.FDKO3, n, 1.0, dt, ko_eps=0.1) for n in (80, 160)]
    assert 3.8 < math.log2(e[0] / e[1]) < 4.3


# --------------------------------------------------------------------------- vacuum


def bloch_from_state(s):
    a, b, cr, ci = s
    return np.array([2 * cr, -2 * ci, a - b]), a + b


def vacuum_state(nz, nv):
    u = np.zeros((2, 4, nz, nv))
    u[:, 0] = 1.0  # pure electron flavour, both species
    return u


@pytest.mark.parametrize("omega,theta", [(0.5, 0.1), (0.1, math.radians(37.0))])
def test_vacuum_oscillation_exact_rk4_map(oracle, omega, theta):
    """mu = 0, z-uniform: each cell's Bloch vector obeys dP/dt = omega B x P with
    B = (sin 2theta, 0, -cos 2theta) (from H_vac of Eq. (ham)); RK4 maps P by
    the stability polynomial of dt A, A x = omega B x x."""
    nz, nv, L = 8, 4, 4.0
    p = oracle.params(nz, nv, L, oracle.FDKO, mu=0.0, omega=omega, theta=theta, cfl=0.4)
    u0 = vacuum_state(nz, nv)
    n = 200
    u = oracle.step(p, u0, n)
    B = np.array([math.sin(2 * theta), 0.0, -math.cos(2 * theta)])
    A = omega * np.array([[0, -B[2], B[1]], [B[2], 0, -B[0]], [-B[1], B[0], 0]])
    M = np.eye(3)
    Z = p.dt * A
    step = np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    for _ in range(n):
        M = step @ M
    P = M @ np.array([0.0, 0.0, 1.0])
    for s in range(2):
        for j in range(nv):
            got, p0 = bloch_from_state(u[s, :, 3, j])
            assert np.max(np.abs(got - P)) < 1e-13
            assert p0 == pytest.approx(1.0, abs=1e-14)


def test_vacuum_closed_form_and_min_survival(oracle):
    """Against Eq. (vac_sols) (error O(dt^4)) and the printed minimum survival
    probability 0.076 for omega = 0.1, theta = 37 degrees (Sec. 4.2)."""
    g = GOLDEN["vacuum_min_survival"]
    omega, theta = g["omega"], math.radians(g["theta_deg"])
    nz, nv, L = 4, 2, 4.0
    dt = 0.5
    p = oracle.params(nz, nv, L, oracle.FDKO, mu=0.0, omega=omega, theta=theta, dt=dt)
    u = vacuum_state(nz, nv)
    t, mins = 0.0, 1.0
    s2, c2 = math.sin(2 * theta), math.cos(2 * theta)
    for _ in range(64):  # 64 x 0.5 = 32 > half period pi/omega
        u = oracle.step(p, u, 1)
        t += dt
        x = math.sin(omega * t / 2) ** 2
        exact = [1 - s2 * s2 * x, s2 * s2 * x, -s2 * c2 * x, 0.5 * s2 * math.sin(omega * t)]
        got = u[0, :, 1, 0]
        assert np.max(np.abs(got - exact)) < 1e-6
        mins = min(mins, got[0])
    assert mins == pytest.approx(g["value"], abs=5e-4)


# --------------------------------------------------------------------------- coupling


def test_hamiltonian_quadrature_equals_moments(oracle):
    nz, nv = 6, 16
    u = inputs.random_state(nz, nv, seed=11)
    pa = oracle.params(nz, nv, 3.0, mu=1.3, omega=0.2, theta=0.3, lam=0.05, hmode=0)
    pb = oracle.params(nz, nv, 3.0, mu=1.3, omega=0.2, theta=0.3, lam=0.05, hmode=1)
    ha, hb = oracle.hamiltonian(pa, u), oracle.hamiltonian(pb, u)
    assert np.max(np.abs(ha - hb)) < 1e-14 * np.max(np.abs(ha))
    ka, kb = oracle.rhs(pa, u), oracle.rhs(pb, u)
    assert np.max(np.abs(ka - kb)) < 1e-13


def test_hamiltonian_structure(oracle):
    """Hbar = H_vac - H_m - H_nunu^*: the nu and nubar Hamiltonians of a beam add up to
    2 H_vac (off-diagonal real parts, diagonal differences) and the imaginary parts agree."""
    nz, nv = 3, 8
    u = inputs.random_state(nz, nv, seed=12)
    om, th, lam = 0.7, 0.4, 0.0
    p = oracle.params(nz, nv, 2.0, mu=2.0, omega=om, theta=th, lam=lam)
    h = oracle.hamiltonian(p, u)
    assert np.allclose(h[0, 0] + h[1, 0], -2 * om * math.cos(2 * th), atol=1e-14)
    assert np.allclose(h[0, 1] + h[1, 1], om * math.sin(2 * th), atol=1e-14)
    assert np.allclose(h[0, 2], h[1, 2], atol=1e-15)
    # the nu-nu part for one beam, written out from Eq. (ham) with numpy
    v, w = oracle.vgrid(nv)
    z, i = 1, 5
    ker = w * (1 - v[i] * v)
    d3 = (u[0, 0, z] - u[0, 1, z]) - (u[1, 0, z] - u[1, 1, z])
    ref = -om * math.cos(2 * th) + 2.0 * np.sum(ker * d3)
    assert h[0, 0, z, i] == pytest.approx(ref, abs=1e-14)
    ref_i = 2.0 * np.sum(ker * (u[0, 3, z] + u[1, 3, z]))
    assert h[0, 2, z, i] == pytest.approx(ref_i, abs=1e-14)


def test_commutator_precession(oracle):
    """z-uniform state: advection vanishes and d/dt of each cell is a commutator, which
    is traceless and orthogonal to the Bloch vector (|P| and P0 are conserved, Sec. 2)."""
    nz, nv = 8, 8
    u1 = inputs.random_state(1, nv, seed=13)
    u = np.repeat(u1, nz, axis=2)
    p = oracle.params(nz, nv, 2.0, mu=1.5, omega=0.3, theta=0.2)
    k = oracle.rhs(p, u)
    for s in range(2):
        P, _ = bloch_from_state(u[s, :, 0, :])
        dP, dP0 = bloch_from_state(k[s, :, 0, :])
        assert np.max(np.abs(dP0)) < 1e-13
        assert np.max(np.abs(np.sum(P * dP, axis=0))) < 1e-13


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_discrete_conservation_laws(oracle, scheme):
    """Periodic z: total traces of both species, the lepton-number vector
    M = sum w dz P(S - Sbar^*) (omega = 0), and its projection on B (omega != 0)
    are conserved by the discrete scheme to round-off (Sec. 5, M_0)."""
    nz, nv = 16, 8
    u0 = inputs.random_state(nz, nv, seed=21)
    p = oracle.params(nz, nv, 5.0, scheme, mu=1.0)
    c0 = oracle.conserved(p, u0)
    c1 = oracle.conserved(p, oracle.step(p, u0, 10))
    for key in ("tr_nu", "tr_nubar"):
        assert c1[key] == pytest.approx(c0[key], rel=1e-13)
    assert np.max(np.abs(c1["M"] - c0["M"])) < 1e-13 * np.max(np.abs(c0["M"]))
    p = oracle.params(nz, nv, 5.0, scheme, mu=1.0, omega=0.8, theta=0.3)
    c1 = oracle.conserved(p, oracle.step(p, u0, 10))
    c0 = oracle.conserved(p, u0)
    assert abs(c1["M_vac"] - c0["M_vac"]) < 1e-13 * np.max(np.abs(c0["M"]))
    assert abs(c1["M"][2] - c0["M"][2]) > 1e-8  # M3 alone is not conserved with omega != 0


def dispersion_growth(nv, k, alpha, sig, sigb, mu=1.0):
    """max Im Omega of the linearised equations for X = S_ex - Sbar_ex^* ~ exp(i(kz - Omega t)):
    Omega X_i = (v_i k + mu (G0 - v_i G1)) X_i - mu G_i sum_j w_j (1 - v_i v_j) X_j."""
    v = inputs.beam_velocities(nv)
    w = np.full(nv, 2.0 / nv)
    G = inputs.angular_gaussian(nv, sig) - alpha * inputs.angular_gaussian(nv, sigb)
    G0, G1 = np.sum(w * G), np.sum(w * v * G)
    M = np.diag(v * k + mu * (G0 - v * G1)) - mu * G[:, None] * (w[None, :] * (1 - np.outer(v, v)))
    return np.max(np.linalg.eigvals(M).imag)


@pytest.mark.slow
def test_fast_instability_growth_rate(oracle):
    """A single-k seed grows at the rate of the linear dispersion relation (within 2%)."""
    fid = GOLDEN["fiducial_collective"]
    nv = 24
    ks = np.linspace(-0.5, 0.5, 201)
    rates = [dispersion_growth(nv, k, fid["alpha"], fid["sigma_nu"], fid["sigma_nubar"]) for k in ks]
    kstar = ks[int(np.argmax(rates))]
    gamma = max(rates)
    assert 0.02 < gamma < 0.08
    nz = 32
    assert kstar < 0  # the fastest mode travels against the forward-peaked beams
    L = 2 * np.pi / abs(kstar)
    p = oracle.params(nz, nv, L, oracle.FDKO, mu=1.0, cfl=0.4)
    u = inputs.single_mode_state(nz, nv, -1, alpha=fid["alpha"], sigma_nu=fid["sigma_nu"],
                                 sigma_nubar=fid["sigma_nubar"], eps0=1e-9)
    T = 220.0
    nchunk = 20
    per = int(round(T / nchunk / p.dt))
    ts, amps = [], []
    for c in range(nchunk):
        u = oracle.step(p, u, per)
        X = (u[0, 2] + 1j * u[0, 3]) - (u[1, 2] - 1j * u[1, 3])
        amps.append(np.linalg.norm(np.fft.fft(X, axis=0)[-1]))
        ts.append((c + 1) * per * p.dt)
    ts, la = np.array(ts), np.log(np.array(amps))
    half = nchunk // 2
    slope = np.polyfit(ts[half:], la[half:], 1)[0]
    # discrete corrections: KO damping of this mode and the FD wavenumber
    h = L / nz
    th = kstar * h
    keff = float(np.imag(fd4_ko_symbol(th, h, -1.0, 0.0)))  # negative, like kstar
    ko_damp = float(np.real(fd4_ko_symbol(th, h, 0.0, 0.1)))
    gamma_d = dispersion_growth(nv, keff, fid["alpha"], fid["sigma_nu"], fid["sigma_nubar"]) + ko_damp
    assert slope == pytest.approx(gamma_d, rel=0.02)
    assert np.max(np.abs(u[:, 2:])) < 1e-3  # still linear: |rho_ex| below 1e-3


# --------------------------------------------------------------------------- diagnostics


def test_conserved_closed_forms(oracle):
    """z- and v-uniform states: every sum is (value) x sum(w dz) = (value) x 2L, and
    |P|/P0 of a cell follows from the Bloch vector P = (2 Re, -2 Im, ee - xx)."""
    nz, nv, L = 5, 8, 3.0
    a, b, cr, ci = 0.7, 0.2, 0.1, -0.15
    ab, bb, cbr, cbi = 0.4, 0.3, -0.05, 0.2
    u = np.zeros((2, 4, nz, nv))
    u[0, 0], u[0, 1], u[0, 2], u[0, 3] = a, b, cr, ci
    u[1, 0], u[1, 1], u[1, 2], u[1, 3] = ab, bb, cbr, cbi
    th = 0.35
    c = oracle.conserved(oracle.params(nz, nv, L, theta=th), u)
    assert c["tr_nu"] == pytest.approx((a + b) * 2 * L, rel=1e-14)
    assert c["tr_nubar"] == pytest.approx((ab + bb) * 2 * L, rel=1e-14)
    M = np.array([2 * (cr - cbr), -2 * (ci + cbi), (a - b) - (ab - bb)]) * 2 * L
    assert np.allclose(c["M"], M, rtol=1e-14, atol=1e-15)
    assert c["M_vac"] == pytest.approx(math.sin(2 * th) * M[0] - math.cos(2 * th) * M[2], abs=1e-14)
    dp_nu = abs(math.sqrt((a - b) ** 2 + 4 * (cr * cr + ci * ci)) / (a + b) - 1)
    dp_nb = abs(math.sqrt((ab - bb) ** 2 + 4 * (cbr * cbr + cbi * cbi)) / (ab + bb) - 1)
    assert c["dP_max"] == pytest.approx(max(dp_nu, dp_nb), rel=1e-13)
    assert c["dP_mean"] == pytest.approx(dp_nu, rel=1e-13)
    # a pure state has |P| = P0
    p = np.zeros((2, 4, nz, nv))
    p[:, 0] = 0.5 * (1 + math.sqrt(1 - 0.3 ** 2))
    p[:, 1] = 0.5 * (1 - math.sqrt(1 - 0.3 ** 2))
    p[:, 2] = 0.15
    assert oracle.conserved(oracle.params(nz, nv, L), p)["dP_max"] < 1e-15


def test_moments_closed_forms(oracle):
    """zavg of cos(2 pi z / nz) + const is const; with S_ee - S_xx = 1 + v the midpoint sums
    give D3_0 = 2 and D3_1 = sum dv v^2 = 2/3 - dv^2/6 (midpoint rule error of v^2)."""
    nz, nv = 8, 16
    z = np.arange(nz)
    v, _ = oracle.vgrid(nv)
    u = np.zeros((2, 4, nz, nv))
    u[0, 0] = (1 + v)[None, :] + np.cos(2 * np.pi * z / nz)[:, None]
    u[0, 1] = np.cos(2 * np.pi * z / nz)[:, None]
    u[1, 2] = 0.25
    u[0, 3] = 0.5 * v[None, :]
    zavg, vmom = oracle.moments(oracle.params(nz, nv, 1.0), u)
    assert np.allclose(zavg[0, 0], 1 + v, atol=1e-15)
    assert np.allclose(zavg[0, 1], 0.0, atol=1e-15)
    assert np.allclose(zavg[1, 2], 0.25, atol=1e-16)
    dv = 2.0 / nv
    assert np.allclose(vmom[:, 0], 2.0, atol=1e-14)
    assert np.allclose(vmom[:, 1], 2.0 / 3.0 - dv * dv / 6.0, atol=1e-14)
    assert np.allclose(vmom[:, 2], -0.25 * 2.0, atol=1e-15)    # Dr = sum dv (cr - cbr)
    assert np.allclose(vmom[:, 3], 0.0, atol=1e-15)
    assert np.allclose(vmom[:, 4], 0.0, atol=1e-15)            # Di_0 = sum dv 0.5 v = 0
    assert np.allclose(vmom[:, 5], 0.5 * (2.0 / 3.0 - dv * dv / 6.0), atol=1e-14)
