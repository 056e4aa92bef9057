"""The seeded input recipes (paper_2203_12866_gb300/inputs.py) that both the oracle
and the CUDA path consume: determinism, ranges and the structure the workloads
state (collective state of Sec. 5, the batched-grid and serving-trace recipes)."""
import numpy as np

from paper_2203_12866_gb300 import inputs


def test_uniform01_is_deterministic_and_in_range():
    a = inputs.uniform01(10000, 12866)
    assert np.array_equal(a, inputs.uniform01(10000, 12866))
    assert not np.array_equal(a, inputs.uniform01(10000, 12867))
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.02 and abs(a.var() - 1.0 / 12.0) < 0.01


def test_collective_state_structure():
    nz, nv, alpha, eps0 = 64, 32, 0.9, 1e-6
    s = inputs.collective_state(nz, nv, alpha=alpha, sigma_nu=0.6, sigma_nubar=0.5, eps0=eps0)
    assert s.shape == (2, 4, nz, nv)
    dv = 2.0 / nv
    # S_ee = g_nu normalised to 1, Sbar_ee = alpha g_nubar, S_xx = Sbar_xx = 0
    assert abs(dv * s[0, 0, 0].sum() - 1.0) < 1e-14
    assert abs(dv * s[1, 0, 0].sum() - alpha) < 1e-14
    assert np.all(s[:, 1] == 0.0)
    # z-independent diagonals, |rho_ex| = eps0 with a seeded random phase shared by both species
    assert np.all(s[:, 0] == s[:, 0, :1])
    amp = np.hypot(s[:, 2], s[:, 3])
    assert np.allclose(amp, eps0, rtol=1e-12)
    assert np.array_equal(s[0, 2:], s[1, 2:])
    assert np.array_equal(s, inputs.collective_state(nz, nv, alpha=alpha, sigma_nu=0.6,
                                                     sigma_nubar=0.5, eps0=eps0))


def test_batch_instances_recipe():
    runs = inputs.batch_instances(256)
    assert runs == inputs.batch_instances(256)
    nz = np.array([r["nz"] for r in runs])
    assert nz.min() >= 1024 and nz.max() <= 32768
    # log-uniform: the median near the geometric mean of the range
    assert 3000 < np.median(nz) < 11000
    assert {r["nv"] for r in runs} == {32, 64, 128}
    assert {r["scheme"] for r in runs} == {0, 1}
    for r in runs:
        assert 0.1 <= r["mu"] <= 10.0
        assert 0.7 <= r["alpha"] <= 1.2
        assert 0.3 <= r["sigma_nu"] <= 0.8 and 0.3 <= r["sigma_nubar"] <= 0.8
        dz = 0.2 / r["mu"]
        assert abs(r["L"] - r["nz"] * dz) < 1e-9 * r["L"]
        assert abs(r["dt"] - 0.4 * dz) < 1e-15 * dz
    assert len({r["seed"] for r in runs}) == 256


def test_serving_trace_recipe():
    tr = inputs.serving_trace(32, 50.0)
    t = np.array([r["t_arrival"] for r in tr])
    assert np.all(np.diff(t) > 0)
    assert 0.3 < t[-1] < 2.0  # 32 arrivals of a rate-50 Poisson process
    assert [r["precision"] for r in tr] == [1 - (i % 2) for i in range(32)]
    for r in tr:
        t_final = r["nsteps"] * r["dt"] * r["mu"]  # in units of 1 / mu
        assert 50.0 - r["dt"] * r["mu"] <= t_final <= 500.0 + r["dt"] * r["mu"]
    scaled = inputs.serving_trace(32, 50.0, step_scale=0.05)
    for a, b in zip(tr, scaled):
        assert abs(b["nsteps"] - 0.05 * a["nsteps"]) <= 1.0
        assert a["t_arrival"] == b["t_arrival"]
