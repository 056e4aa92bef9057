"""The float WENO7 path evaluates the smoothness indicators of Eq. (Si4) as sums
of squares of one-sided differences (stage_kernel.cuh, weno7_si_sos).  That form
must equal the printed quadratic forms exactly; checked here in exact rational
arithmetic on random integer data and on the basis vectors (which fixes every
coefficient of the quadratic form)."""
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
