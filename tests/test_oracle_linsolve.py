"""Prop. 3 (closed-form AA^T solve) against a dense direct solve."""
import numpy as np
import pytest

from oracle import reduced_model as rm
from oracle.linsolve import solve_aat


@pytest.mark.parametrize("m,n", [(2, 2), (3, 3), (4, 5), (5, 4), (8, 8), (2, 7), (7, 2), (6, 3)])
def test_prop3_equals_dense_solve(m, n):
    A = rm.build_A(m, n)
    AAt = (A @ A.T).toarray()
    rng = np.random.default_rng(m * 100 + n)
    for _ in range(3):
        R = rng.standard_normal(3 * m * n - 1) * 10.0 ** rng.integers(-3, 3)
        y = solve_aat(R, m, n)
        y_ref = np.linalg.solve(AAt, R)
        scale = np.abs(y_ref).max()
        assert np.abs(y - y_ref).max() <= 1e-12 * scale
        assert np.abs(AAt @ y - R).max() <= 1e-12 * np.abs(R).max() * (m + n)


def test_prop3_is_linear_and_exact_on_basis_vectors():
    m, n = 3, 4
    A = rm.build_A(m, n)
    AAt = (A @ A.T).toarray()
    Y = np.column_stack([solve_aat(e, m, n) for e in np.eye(3 * m * n - 1)])
    np.testing.assert_allclose(AAt @ Y, np.eye(3 * m * n - 1), atol=1e-13)
