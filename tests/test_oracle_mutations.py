"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case copies one oracle step with a plausible slip (a dropped term, a
wrong sign, a swapped operand) and shows that the corresponding pin fails."""
import numpy as np

from oracle import hot, linsolve
from oracle import reduced_model as rm
from paper_2408_00598_gb300 import synthetic as syn


def _state(m=4, n=5, seed=3):
    rng = np.random.default_rng(seed)
    mu1, mu2 = syn.make_pair("gauss", m, seed, n)
    A = rm.build_A(m, n)
    b = rm.build_b(mu1, mu2)
    c = rm.build_c(m, n) / hot.cost_scale(rm.build_c(m, n))
    x = rng.standard_normal(c.size) * 0.01
    z = np.abs(rng.standard_normal(c.size))
    return A, b, c, x, z, m, n


def _prop3_error(solver, m, n):
    A = rm.build_A(m, n)
    R = np.random.default_rng(0).standard_normal(3 * m * n - 1)
    return np.abs(solver(R, m, n) - np.linalg.solve((A @ A.T).toarray(), R)).max()


def test_dropping_the_low_rank_correction_is_caught():
    """Prop. 3 without the y1^a term (W-hat taken as 0) fails the dense pin."""
    def bad(R, m, n):
        R1, R2, R3 = linsolve.split_blocks(R, m, n)
        one = np.ones(m)
        Ibar = np.eye(m)[: m - 1]
        sumR3 = sum(R3[j] for j in range(n - 1)) + Ibar.T @ R3[n - 1]
        Rt3 = sumR3 / n + sum(float(np.sum(r)) for r in R3) / n ** 2
        y1 = [(R1[j] + (one @ R1[j]) / n * one - (1 / m + 1 / n) * (one @ R2[j]) * one + Rt3) / (m + n)
              for j in range(n)]                                   # planted: y1 = y1-hat
        y2 = [(R2[j] - (one @ y1[j]) * one) / m for j in range(n)]
        s = sum(y1)
        y3 = [(R3[j] + s) / n for j in range(n - 1)] + [(R3[n - 1] + Ibar @ s) / n]
        return np.concatenate(y1 + y2 + y3)
    assert _prop3_error(linsolve.solve_aat, 4, 5) < 1e-12
    assert _prop3_error(bad, 4, 5) > 1e-6


def test_garbled_y3_reading_is_caught():
    """Reading y3^j with only y1^j instead of the sum over all blocks fails the dense pin."""
    def bad(R, m, n):
        y = linsolve.solve_aat(R, m, n).copy()
        M = m * n
        y1 = y[:M].reshape(n, m)
        R3 = np.concatenate([R[2 * M:], [0.0]]).reshape(n, m)
        y3 = (R3 + y1) / n                       # wrong: y1^j instead of sum_j y1^j
        y[2 * M:] = y3.reshape(-1)[:M - 1]
        return y
    assert _prop3_error(bad, 4, 5) > 1e-6


def test_sign_slip_in_step2_is_caught():
    A, b, c, x, z, m, n = _state()
    sigma = 0.2
    y_bar, x_bar, z_bar = hot.hot_step(A, b, c, sigma, x, z, m, n)
    assert np.abs(A @ x_bar - b).max() < 1e-13
    x_bad = x - sigma * (A.T @ y_bar + z - c)        # planted: wrong sign
    assert np.abs(A @ x_bad - b).max() > 1e-6


def test_wrong_projection_in_step3_is_caught():
    A, b, c, x, z, m, n = _state()
    sigma = 0.2
    y_bar, x_bar, z_bar = hot.hot_step(A, b, c, sigma, x, z, m, n)
    z_bad = np.minimum(c - A.T @ y_bar - x_bar / sigma, 0.0)   # planted: min for max
    xt = x_bar + sigma * (A.T @ y_bar + z_bad - c)
    assert xt.min() < -1e-6 or z_bad.min() < 0


def test_transposed_f2_layout_is_caught():
    """Storing f2 as [k][j][l] in the paper's vector (instead of [l][j][k])
    breaks the meaning check of eq. (3)."""
    m, n = 3, 4
    rng = np.random.default_rng(2)
    pi = rng.random((m, n, m, n))
    pi /= pi.sum()
    mu1, mu2 = pi.sum(axis=(2, 3)), pi.sum(axis=(0, 1))
    f1 = np.einsum("ijkl->ikj", pi)
    f2 = np.einsum("ijkl->kjl", pi)
    good = np.concatenate([f1.transpose(2, 1, 0).reshape(-1), f2.transpose(2, 1, 0).reshape(-1)])
    bad = np.concatenate([f1.transpose(2, 1, 0).reshape(-1), f2.reshape(-1)])
    A, b = rm.build_A(m, n), rm.build_b(mu1, mu2)
    assert np.abs(A @ good - b).max() < 1e-14
    assert np.abs(A @ bad - b).max() > 1e-4
