"""Seeded synthetic initial states (host numpy arrays, FP64).

This module only builds inputs; it contains none of the solver's arithmetic.
Both the CUDA path and the CPU oracle receive the arrays it returns, so
neither side draws random numbers of its own.

State layout: float64 [2 species][4 components][nz][nv], species (nu, nubar),
components (rho_ee, rho_xx, Re rho_ex, Im rho_ex), v fastest.

Recipe of the collective-oscillation runs (Sec. 5 of arXiv:2203.12866):
  * angular distributions g(v) proportional to exp(-(v-1)^2 / (2 sigma^2)), Sec. 5,
    normalised on the grid (sum_j w_j g_j = 1 with midpoint bins, w_j = 2/nv);
  * neutrino state S_ee = g_nu, S_xx = 0; antineutrino state carries alpha:
    Sbar_ee = alpha g_nubar, Sbar_xx = 0;
  * off-diagonal seed S_ex = Sbar_ex = eps0 exp(i phi(z)), phi(z_i) uniform
    on [0, 2 pi) drawn per cell by splitmix64(seed XOR i); u = (x >> 11) 2^-53.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    x = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(_M64)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def uniform01(n: int, seed: int) -> np.ndarray:
    """n doubles in [0, 1): (splitmix64(seed ^ i) >> 11) * 2^-53."""
    with np.errstate(over="ignore"):
        i = np.arange(n, dtype=np.uint64) ^ np.uint64(seed & _M64)
        x = splitmix64(i)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def beam_velocities(nv: int) -> np.ndarray:
    """Bin midpoints on [-1, 1] (where the angular distributions are sampled)."""
    return -1.0 + (np.arange(nv) + 0.5) * (2.0 / nv)


def angular_gaussian(nv: int, sigma: float) -> np.ndarray:
    """g(v) ~ exp(-(v-1)^2/(2 sigma^2)) sampled at bin midpoints, sum(w g) = 1."""
    v = beam_velocities(nv)
    g = np.exp(-((v - 1.0) ** 2) / (2.0 * sigma * sigma))
    return g / (g.sum() * (2.0 / nv))


def collective_state(nz: int, nv: int, *, alpha=0.9, sigma_nu=0.6, sigma_nubar=0.5,
                     eps0=1e-6, seed=12866) -> np.ndarray:
    """Initial state of the collective runs with a random-phase seed."""
    g = angular_gaussian(nv, sigma_nu)
    gb = angular_gaussian(nv, sigma_nubar)
    phi = 2.0 * np.pi * uniform01(nz, seed)
    s = np.zeros((2, 4, nz, nv))
    s[0, 0] = g[None, :]
    s[1, 0] = alpha * gb[None, :]
    for sp in range(2):
        s[sp, 2] = (eps0 * np.cos(phi))[:, None]
        s[sp, 3] = (eps0 * np.sin(phi))[:, None]
    return s


def random_state(nz: int, nv: int, seed: int, scale=1.0, offdiag=0.1) -> np.ndarray:
    """Generic seeded state for parity tests: diagonal in [0.5, 1.5) * scale,
    off-diagonal uniform in [-offdiag, offdiag) * scale."""
    u = uniform01(8 * nz * nv, seed).reshape(2, 4, nz, nv)
    s = np.empty_like(u)
    s[:, 0:2] = (0.5 + u[:, 0:2]) * scale
    s[:, 2:4] = (2.0 * u[:, 2:4] - 1.0) * offdiag * scale
    return s


def single_mode_state(nz: int, nv: int, k_index: int, *, alpha=0.9, sigma_nu=0.6,
                      sigma_nubar=0.5, eps0=1e-8) -> np.ndarray:
    """Collective state seeded with one Fourier mode exp(i k z), k = 2 pi k_index / L,
    on the neutrino off-diagonal only."""
    s = collective_state(nz, nv, alpha=alpha, sigma_nu=sigma_nu, sigma_nubar=sigma_nubar,
                         eps0=0.0)
    ph = 2.0 * np.pi * k_index * np.arange(nz) / nz
    s[0, 2] = (eps0 * np.cos(ph))[:, None]
    s[0, 3] = (eps0 * np.sin(ph))[:, None]
    return s


def collective_rows(z_index: np.ndarray, nv: int, *, alpha=0.9, sigma_nu=0.6, sigma_nubar=0.5,
                    eps0=1e-6, seed=12866) -> np.ndarray:
    """Rows z_index (any integers, taken as given) of collective_state(): the same
    values without building the whole grid.  Shape [2][4][len(z_index)][nv]."""
    z_index = np.asarray(z_index, dtype=np.int64)
    g = angular_gaussian(nv, sigma_nu)
    gb = angular_gaussian(nv, sigma_nubar)
    n = int(z_index.max()) + 1 if z_index.size else 0
    phi = 2.0 * np.pi * uniform01(n, seed)[z_index]
    s = np.zeros((2, 4, z_index.size, nv))
    s[0, 0] = g[None, :]
    s[1, 0] = alpha * gb[None, :]
    for sp in range(2):
        s[sp, 2] = (eps0 * np.cos(phi))[:, None]
        s[sp, 3] = (eps0 * np.sin(phi))[:, None]
    return s


def collective_state_device(nz: int, nv: int, device, *, alpha=0.9, sigma_nu=0.6,
                            sigma_nubar=0.5, eps0=1e-6, seed=12866):
    """collective_state() built on a torch device from the same host-computed
    vectors (g(v), eps0 cos phi(z), eps0 sin phi(z)); the device only broadcasts,
    so the values are bit-identical to the host version."""
    import torch

    g = torch.from_numpy(angular_gaussian(nv, sigma_nu)).to(device)
    gb = torch.from_numpy(alpha * angular_gaussian(nv, sigma_nubar)).to(device)
    phi = 2.0 * np.pi * uniform01(nz, seed)
    cr = torch.from_numpy(eps0 * np.cos(phi)).to(device)
    ci = torch.from_numpy(eps0 * np.sin(phi)).to(device)
    s = torch.zeros((2, 4, nz, nv), dtype=torch.float64, device=device)
    s[0, 0] = g[None, :]
    s[1, 0] = gb[None, :]
    for sp in range(2):
        s[sp, 2] = cr[:, None]
        s[sp, 3] = ci[:, None]
    return s


def batch_instances(n: int, *, seed=12866, nz_range=(1024, 32768), nv_choices=(32, 64, 128),
                    mu_range=(0.1, 10.0), alpha_range=(0.7, 1.2), sigma_range=(0.3, 0.8),
                    schemes=(0, 1), dz_mu=0.2, cfl=0.4):
    """Parameters of n independent collective-oscillation grids for the batched
    solver: nz log-uniform on nz_range, nv uniform over nv_choices, mu
    log-uniform on mu_range, alpha and both sigmas uniform, scheme uniform over
    `schemes`; dz = dz_mu / mu, L = nz dz, dt = cfl dz.  Each parameter draws
    from its own uniform01 stream (seed + k); instance i's state seed is
    seed + 1000 + i.  Returns a list of dicts."""
    u = [uniform01(n, seed + k) for k in range(7)]
    lo, hi = np.log(nz_range[0]), np.log(nz_range[1])
    out = []
    for i in range(n):
        nz = int(np.floor(np.exp(lo + (hi - lo) * u[0][i])))
        nv = int(nv_choices[min(int(u[1][i] * len(nv_choices)), len(nv_choices) - 1)])
        mu = float(np.exp(np.log(mu_range[0]) + np.log(mu_range[1] / mu_range[0]) * u[2][i]))
        alpha = alpha_range[0] + (alpha_range[1] - alpha_range[0]) * u[3][i]
        s_nu = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * u[4][i]
        s_nb = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * u[5][i]
        scheme = int(schemes[min(int(u[6][i] * len(schemes)), len(schemes) - 1)])
        dz = dz_mu / mu
        out.append({"nz": nz, "nv": nv, "mu": mu, "alpha": float(alpha), "sigma_nu": float(s_nu),
                    "sigma_nubar": float(s_nb), "scheme": scheme, "L": nz * dz, "dt": cfl * dz,
                    "seed": seed + 1000 + i})
    return out


def serving_trace(n: int, rate: float, *, seed=12866, step_scale=1.0, **grid_kw):
    """A trace of n runs for the serving loop: arrival times of a Poisson process
    of `rate` runs per second (exponential gaps -ln(1 - u) / rate from uniform01
    stream seed + 100), grids from batch_instances(n, seed=seed, **grid_kw),
    precision alternating mixed / FP64 (run i: mixed if i is even), and a final
    time t_final = U[50, 500] / mu (stream seed + 101) turned into
    nsteps = max(1, round(step_scale * t_final / dt)).  Returns a list of dicts
    (the batch_instances fields plus t_arrival, precision, nsteps)."""
    runs = batch_instances(n, seed=seed, **grid_kw)
    gaps = -np.log1p(-uniform01(n, seed + 100)) / rate
    tf = uniform01(n, seed + 101)
    t = 0.0
    for i, r in enumerate(runs):
        t += float(gaps[i])
        r["t_arrival"] = t
        r["precision"] = 1 if i % 2 == 0 else 0
        t_final = (50.0 + 450.0 * float(tf[i])) / r["mu"]
        r["nsteps"] = max(1, int(round(step_scale * t_final / r["dt"])))
    return runs


def gaussian_perturbation_state(nz: int, nv: int, L: float, *, alpha=0.9, sigma_nu=0.6,
                                sigma_nubar=0.5, amp=1e-2, width2=50.0) -> np.ndarray:
    """Initial state of the collective-oscillation test of Sec. 5 with the paper's
    own perturbation (Eqs. (pert_ee), (pert_xx), (pert_ex)): at cell centres
    z_i = -L/2 + (i + 1/2) L/nz, eps(z) = amp exp(-z^2 / width2) and
    rho_ee = (1 + sqrt(1 - eps^2)) / 2, rho_xx = (1 - sqrt(1 - eps^2)) / 2,
    rho_ex = eps / 2 (real), the same for rhobar; stored as S = g_nu rho and
    Sbar = alpha g_nubar rhobar."""
    dz = L / nz
    z = -L / 2 + (np.arange(nz) + 0.5) * dz
    eps = amp * np.exp(-z * z / width2)
    root = np.sqrt(1.0 - eps * eps)
    rho = [(1.0 + root) / 2.0, (1.0 - root) / 2.0, eps / 2.0, np.zeros(nz)]
    g = [angular_gaussian(nv, sigma_nu), alpha * angular_gaussian(nv, sigma_nubar)]
    s = np.empty((2, 4, nz, nv))
    for sp in range(2):
        for c in range(4):
            s[sp, c] = rho[c][:, None] * g[sp][None, :]
    return s
