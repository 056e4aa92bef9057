"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/cosenu_oracle.c (on the CPU),
builds it, and runs the pin tests against it: at least one pin must fail.
"""
import os

import pytest

import oracle as oracle_mod
import test_oracle_pins as pins

MUTATIONS = {
    "KO added with the printed sign": (
        "adv = -vg[j] * dudz - Qu;", "adv = -vg[j] * dudz + Qu;"),
    "FD4 denominator": (
        "(um2 - 8.0 * um1 + 8.0 * up1 - up2) / (12.0 * h)",
        "(um2 - 8.0 * um1 + 8.0 * up1 - up2) / (10.0 * h)"),
    "WENO linear weights in the printed order": (
        "const double d[4] = {4.0 / 35.0, 18.0 / 35.0, 12.0 / 35.0, 1.0 / 35.0};",
        "const double d[4] = {1.0 / 35.0, 12.0 / 35.0, 18.0 / 35.0, 4.0 / 35.0};"),
    "WENO smoothness coefficient": ("+ fp1 * (11003.0 * fp1", "+ fp1 * (11004.0 * fp1"),
    "WENO mirror for v < 0": (
        "const int64_t src = vg[j] > 0.0 ? i + m : i + 1 - m;",
        "const int64_t src = vg[j] > 0.0 ? i + m : i - m;"),
    "Hbar with + H_nunu^*": (
        "hb[e] = hvac[a][b] - hmat[a][b] - p->mu * conj(hnn[e]);",
        "hb[e] = hvac[a][b] - hmat[a][b] + p->mu * conj(hnn[e]);"),
    "commutator sign": ("C[r * 2 + c] = -I * (hr - rh);", "C[r * 2 + c] = I * (hr - rh);"),
    "kernel 1 + v v'": ("for (int e = 0; e < 4; ++e) hnn[e] = m0[e] - vg[i] * m1[e];",
                        "for (int e = 0; e < 4; ++e) hnn[e] = m0[e] + vg[i] * m1[e];"),
    "Sbar not conjugated": ("cplx d = r[e] - conj(rb[e]);", "cplx d = r[e] - rb[e];"),
    "RK4 weight of k2": ("(k1[e] + 2.0 * k2[e] + 2.0 * k3[e] + k4[e])",
                         "(k1[e] + k2[e] + 2.0 * k3[e] + k4[e])"),
    "left-endpoint velocity bins": ("v[j] = -1.0 + j * dv + 0.5 * dv;", "v[j] = -1.0 + j * dv;"),
    "KO r = 3 normalisation 2^6": ("(h * h * h * h * h) * dd[0] / 64.0;",
                                   "(h * h * h * h * h) * dd[0] / 32.0;"),
    "KO r = 3 sign (-1)^3": ("Qu = p->ko_eps * -1.0 /* (-1)^3 */", "Qu = p->ko_eps * 1.0 /* (-1)^3 */"),
    "Simpson 3/8 end panel weight": ("    w[n - 2] += 9.0 * h / 8.0;", "    w[n - 2] += 8.0 * h / 8.0;"),
    "M2 sign": ("M[1] += wg[j] * h * (P[0][2] + P[1][2]);",
                "M[1] += wg[j] * h * (P[0][2] - P[1][2]);"),
}

PINS = [
    (pins.test_vgrid_midpoints, {}),
    (pins.test_vgrid_vertex_quadratures, {"nv": 12}),
    (pins.test_weno7_constant_data, {}),
    (pins.test_weno7_cubic_reconstructed_exactly, {"seed": 1}),
    (pins.test_weno7_linear_weights_reproduce_eq_f7, {}),
    (pins.test_weno7_smoothness_index_is_scaled_jiang_shu, {"seed": 0}),
    (pins.test_weno7_weight_formula, {}),
    (pins.test_fdko_pure_advection_equals_dft_solution, {"ko_eps": 0.1}),
    (pins.test_fdko3_pure_advection_equals_dft_solution, {"ko_eps": 0.1}),
    (pins.test_weno7_linear_limit_equals_dft_solution, {}),
    (pins.test_vacuum_oscillation_exact_rk4_map, {"omega": 0.5, "theta": 0.1}),
    (pins.test_hamiltonian_structure, {}),
    (pins.test_commutator_precession, {}),
    (pins.test_discrete_conservation_laws, {"scheme": 0}),
    (pins.test_conserved_closed_forms, {}),
    (pins.test_moments_closed_forms, {}),
    (pins.test_fast_instability_growth_rate, {}),
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(oracle_mod.SOURCE).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    mutant = oracle_mod.OracleLib(oracle_mod.compile_source(str(path), str(tmp_path / "m.so")))
    failed = []
    for fn, kw in PINS:
        try:
            fn(mutant, **kw)
        except AssertionError:
            failed.append(fn.__name__)
    assert failed, f"no pin caught: {name}"


def test_unmutated_oracle_passes_the_same_pins():
    ok = oracle_mod.OracleLib(oracle_mod.build())
    for fn, kw in PINS:
        fn(ok, **kw)
