"""Pin of the oracle's relative KKT residual, eq. (kkt_res) of Sec. IV-A:

    max{ ||A^T y + z - c|| / (1 + ||c||),
         ||min(x, z)||     / (1 + ||x|| + ||z||),
         ||A x - b||       / (1 + ||b||) }.

A hand-worked example on a 2 x 3 matrix whose three terms have closed forms
(Pythagorean norms), chosen so that every "1 +" normaliser changes the answer:
||b|| != ||c||, ||z|| != 0 and ||x|| != ||z||, and each of the three terms
can be made the largest.  The expected values below are worked out by hand in
the comments, not by re-running the formula.
"""
import math

import numpy as np
import pytest

from oracle import hot

# A = [[1, 0, 1],
#      [0, 1, 1]]
A = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
b = np.array([6.0, 8.0])          # ||b|| = 10
c = np.array([2.0, 2.0, 1.0])     # ||c|| = 3
y = np.array([1.0, 1.0])          # A^T y = (1, 1, 2)
z = np.array([1.0, 1.0, 1.0])     # ||z|| = sqrt(3)
x = np.array([3.0, 0.0, 4.0])     # ||x|| = 5, A x = (7, 4)

# dual:   A^T y + z - c = (1+1-2, 1+1-2, 2+1-1) = (0, 0, 2)  -> 2 / (1 + 3) = 1/2
DUAL = 0.5
# comp:   min(x, z) = (1, 0, 1) -> sqrt(2) / (1 + 5 + sqrt(3))
COMP = math.sqrt(2.0) / (6.0 + math.sqrt(3.0))
# primal: A x - b = (7 - 6, 4 - 8) = (1, -4) -> sqrt(17) / (1 + 10) = sqrt(17)/11
PRIMAL = math.sqrt(17.0) / 11.0


def test_each_term_of_the_relative_residual_by_hand():
    err, parts = hot.kkt_residual(A, b, c, x, y, z)
    assert parts[0] == pytest.approx(DUAL, rel=1e-15)
    assert parts[1] == pytest.approx(COMP, rel=1e-15)
    assert parts[2] == pytest.approx(PRIMAL, rel=1e-15)
    assert err == pytest.approx(max(DUAL, COMP, PRIMAL), rel=1e-15)
    assert err == pytest.approx(0.5, rel=1e-15)          # the dual term is the largest here


def test_example_separates_the_plausible_mistakes():
    """The hand example is only a pin if the likely slips give other numbers."""
    err, parts = hot.kkt_residual(A, b, c, x, y, z)
    wrong = {
        "||c|| in the primal denominator": math.sqrt(17.0) / (1.0 + 3.0),     # 1.03
        "||b|| in the dual denominator": 2.0 / (1.0 + 10.0),                  # 0.18
        "no ||z|| in the complementarity denominator": math.sqrt(2.0) / 6.0,  # 0.236
        "no ||x|| in the complementarity denominator": math.sqrt(2.0) / (1.0 + math.sqrt(3.0)),
        "no 1 + in the dual denominator": 2.0 / 3.0,
        "no 1 + in the primal denominator": math.sqrt(17.0) / 10.0,
        "squared norms (primal)": 17.0 / 11.0,
        "1-norm (primal)": 5.0 / 11.0,
    }
    got = {"dual": parts[0], "comp": parts[1], "primal": parts[2]}
    for what, v in wrong.items():
        key = "primal" if "primal" in what else ("comp" if "complementarity" in what else "dual")
        assert abs(got[key] - v) > 1e-3, what


@pytest.mark.parametrize("scale_x,expect", [
    # x = t (3, 0, 4): A x - b = (7t - 6, 4t - 8); at t = 4: (22, 8), ||.|| = sqrt(548)
    # -> primal = sqrt(548) / 11 = 2.128; comp = ||min(4x, z)|| = ||(1, 0, 1)|| = sqrt(2),
    #    over 1 + 20 + sqrt(3) -> 0.0622; dual unchanged 0.5  => primal is the largest
    (4.0, math.sqrt(548.0) / 11.0),
])
def test_primal_term_can_dominate(scale_x, expect):
    err, parts = hot.kkt_residual(A, b, c, scale_x * x, y, z)
    assert parts[1] == pytest.approx(math.sqrt(2.0) / (21.0 + math.sqrt(3.0)), rel=1e-15)
    assert err == pytest.approx(expect, rel=1e-15)


def test_complementarity_term_can_dominate():
    # y = (1, 1), z = (2, 2, 2)... keep the dual term small: z = c - A^T y + (0, 0, 0) is
    # not >= 0 here, so take c' = A^T y + z = (3, 3, 4) with z = (2, 2, 2): dual = 0.
    # x = (2, 2, 2): min(x, z) = (2, 2, 2), ||.|| = sqrt(12); ||x|| = ||z|| = sqrt(12)
    # -> comp = sqrt(12) / (1 + 2 sqrt(12)) = 0.4645; A x = (4, 4), b' = (4, 4): primal 0
    cc = np.array([3.0, 3.0, 4.0])
    zz = np.array([2.0, 2.0, 2.0])
    xx = np.array([2.0, 2.0, 2.0])
    bb = np.array([4.0, 4.0])
    err, parts = hot.kkt_residual(A, bb, cc, xx, y, zz)
    assert parts[0] == 0.0 and parts[2] == 0.0
    assert err == pytest.approx(math.sqrt(12.0) / (1.0 + 2.0 * math.sqrt(12.0)), rel=1e-15)


def test_absolute_residual_of_the_same_example():
    # Table VI: the three norms without normalisers: max(2, sqrt(2), sqrt(17)) = sqrt(17)
    assert hot.kkt_absolute(A, b, c, x, y, z) == pytest.approx(math.sqrt(17.0), rel=1e-15)
