"""The WENO7 kernels (both precisions) evaluate the smoothness indicators of
Eq. (Si4) as sums of squares, and both the indicators and the candidate values of
Eq. (f4s) in the first, second and third differences of the seven cell values,
with the linear weights folded into the candidates' coefficients
(stage_kernel.cuh: weno7_face for FP64, weno7_face_core / weno7_face_pair
for float).  Those forms must equal the printed ones exactly; checked
here in exact rational arithmetic on random integer data and on the basis
vectors (which fixes every coefficient of the linear and quadratic forms)."""
from fractions import Fraction as F

import numpy as np


def printed(f):
    fm3, fm2, fm1, f0, fp1, fp2, fp3 = f
    return [
        f0 * (2107 * f0 - 9402 * fp1 + 7042 * fp2 - 1854 * fp3) + fp1 * (
            11003 * fp1 - 17246 * fp2 + 4642 * fp3) + fp2 * (7043 * fp2 - 3882 * fp3)
        + 547 * fp3 * fp3,
        fm1 * (547 * fm1 - 2522 * f0 + 1922 * fp1 - 494 * fp2) + f0 * (
            3443 * f0 - 5966 * fp1 + 1602 * fp2) + fp1 * (2843 * fp1 - 1642 * fp2)
        + 267 * fp2 * fp2,
        fm2 * (267 * fm2 - 1642 * fm1 + 1602 * f0 - 494 * fp1) + fm1 * (
            2843 * fm1 - 5966 * f0 + 1922 * fp1) + f0 * (3443 * f0 - 2522 * fp1)
        + 547 * fp1 * fp1,
        fm3 * (547 * fm3 - 3882 * fm2 + 4642 * fm1 - 1854 * f0) + fm2 * (
            7043 * fm2 - 17246 * fm1 + 7042 * f0) + fm1 * (11003 * fm1 - 9402 * f0)
        + 2107 * f0 * f0]


def sums_of_squares(f):
    fm3, fm2, fm1, f0, fp1, fp2, fp3 = f
    c1, c2, c3 = F(20, 3), F(260), F(781, 3)
    a = [-11 * f0 + 18 * fp1 - 9 * fp2 + 2 * fp3, -2 * fm1 - 3 * f0 + 6 * fp1 - fp2,
         fm2 - 6 * fm1 + 3 * f0 + 2 * fp1, -2 * fm3 + 9 * fm2 - 18 * fm1 + 11 * f0]
    b = [2 * f0 - 5 * fp1 + 4 * fp2 - fp3, fm1 - 2 * f0 + fp1, fm1 - 2 * f0 + fp1,
         2 * f0 - 5 * fm1 + 4 * fm2 - fm3]
    c = [-f0 + 3 * fp1 - 3 * fp2 + fp3, -fm1 + 3 * f0 - 3 * fp1 + fp2,
         -fm2 + 3 * fm1 - 3 * f0 + fp1, -fm3 + 3 * fm2 - 3 * fm1 + f0]
    return [c1 * a[k] ** 2 + c2 * b[k] ** 2 + c3 * c[k] ** 2 for k in range(4)]


def test_sum_of_squares_equals_printed_forms():
    rng = np.random.default_rng(2203)
    cases = [[F(int(x)) for x in rng.integers(-50, 51, 7)] for _ in range(200)]
    for i in range(7):
        for j in range(7):  # e_i + e_j spans every monomial of the quadratic form
            v = [F(0)] * 7
            v[i] += 1
            v[j] += 1
            cases.append(v)
    for f in cases:
        assert sums_of_squares(f) == printed(f)


def printed_candidates(f):
    fm3, fm2, fm1, f0, fp1, fp2, fp3 = f
    return [(3 * f0 + 13 * fp1 - 5 * fp2 + fp3) / 12, (-fm1 + 7 * f0 + 7 * fp1 - fp2) / 12,
            (fm2 - 5 * fm1 + 13 * f0 + 3 * fp1) / 12, (-3 * fm3 + 13 * fm2 - 23 * fm1 + 25 * f0) / 12]


def difference_form(f):
    """The kernel's arrangement: e_k = f_{k+1} - f_k, g_k = e_{k+1} - e_k,
    h_k = g_{k+1} - g_k; candidates f_0 + delta_r; SI_r from (a_r, b_r, c_r)."""
    fm3, fm2, fm1, f0, fp1, fp2, fp3 = f
    em3, em2, em1, e0, e1, e2 = fm2 - fm3, fm1 - fm2, f0 - fm1, fp1 - f0, fp2 - fp1, fp3 - fp2
    gm3, gm2, gm1, g0, g1 = em2 - em3, em1 - em2, e0 - em1, e1 - e0, e2 - e1
    hm3, hm2, hm1, h0 = gm2 - gm3, gm1 - gm2, g0 - gm1, g1 - g0
    c1, c2, c3 = F(20, 3), F(260), F(781, 3)
    a = [11 * e0 - 7 * e1 + 2 * e2, 2 * em1 + 5 * e0 - e1, -em2 + 5 * em1 + 2 * e0,
         2 * em3 - 7 * em2 + 11 * em1]
    b = [2 * g0 - g1, gm1, gm1, 2 * gm2 - gm3]
    c = [h0, hm1, hm2, hm3]
    si = [c1 * a[k] ** 2 + c2 * b[k] ** 2 + c3 * c[k] ** 2 for k in range(4)]
    delta = [F(3, 4) * e0 - F(1, 3) * e1 + F(1, 12) * e2,
             F(1, 12) * em1 + F(1, 2) * e0 - F(1, 12) * e1,
             -F(1, 12) * em2 + F(1, 3) * em1 + F(1, 4) * e0,
             F(1, 4) * em3 - F(5, 6) * em2 + F(13, 12) * em1]
    dd = [F(3, 35) * e0 - F(4, 105) * e1 + F(1, 105) * e2,
          F(3, 70) * em1 + F(9, 35) * e0 - F(3, 70) * e1,
          -F(1, 35) * em2 + F(4, 35) * em1 + F(3, 35) * e0,
          F(1, 140) * em3 - F(1, 42) * em2 + F(13, 420) * em1]
    return [f0 + d for d in delta], si, dd


def _cases():
    rng = np.random.default_rng(2204)
    cases = [[F(int(x)) for x in rng.integers(-50, 51, 7)] for _ in range(200)]
    for i in range(7):
        for j in range(7):
            v = [F(0)] * 7
            v[i] += 1
            v[j] += 1
            cases.append(v)
    return cases


def test_difference_form_equals_printed_forms():
    for f in _cases():
        cand, si, dd = difference_form(f)
        assert cand == printed_candidates(f)
        assert si == printed(f)
        # linear weights of Eq. (weight) folded into the candidates
        d = [F(4, 35), F(18, 35), F(12, 35), F(1, 35)]
        assert dd == [d[r] * (cand[r] - f[3]) for r in range(4)]


def test_difference_form_catches_a_wrong_coefficient():
    # the check above is not vacuous: one coefficient off by one is detected
    f = [F(x) for x in (3, -1, 4, 1, -5, 9, 2)]
    cand, si, dd = difference_form(f)
    fm3, fm2, fm1, f0, fp1, fp2, fp3 = f
    em2, em1, e0 = fm1 - fm2, f0 - fm1, fp1 - f0
    wrong = -F(1, 12) * em2 + F(1, 3) * em1 + F(1, 3) * e0 + f0
    assert wrong != printed_candidates(f)[2] and cand[2] == printed_candidates(f)[2]
