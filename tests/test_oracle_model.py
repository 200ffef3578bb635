"""Pins of the oracle's model data (eq. 3-8 and eq. Mat:OT_AAT of arXiv 2408.00598)."""
import numpy as np
import pytest

from oracle import reduced_model as rm

SHAPES = [(2, 2), (3, 3), (3, 4), (4, 3), (5, 2), (2, 5)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_aat_matches_printed_blocks(m, n):
    """A A^T from the Kronecker blocks of eq. (6)-(8) equals the block matrix of
    eq. (Mat:OT_AAT) built from E1..E5 as printed: two separate definitions."""
    A = rm.build_A(m, n)
    lhs = (A @ A.T).toarray()
    rhs = rm.aat_from_blocks(m, n)
    assert lhs.shape == (3 * m * n - 1, 3 * m * n - 1)
    np.testing.assert_array_equal(lhs, rhs)


@pytest.mark.parametrize("m,n", SHAPES)
def test_A_full_row_rank_and_same_feasible_set(m, n):
    """A has full row rank and {Ax = b} = {A-hat x = b-hat} (text after eq. 8)."""
    A = rm.build_A(m, n)
    Ah = rm.build_A_hat(m, n)
    assert np.linalg.matrix_rank(A.toarray()) == 3 * m * n - 1
    assert np.linalg.matrix_rank(Ah.toarray()) == 3 * m * n - 1
    # the dropped row of A-hat is a combination of the rows of A
    sol, *_ = np.linalg.lstsq(A.toarray().T, Ah.toarray()[-1], rcond=None)
    np.testing.assert_allclose(A.toarray().T @ sol, Ah.toarray()[-1], atol=1e-12)


def _flows_from_plan(pi, m, n):
    """Route pi_{ij;kl} through the intermediate node (k, j) as in eq. (3):
    f1_{i,k,j} = sum_l pi, f2_{k,j,l} = sum_i pi."""
    f1 = np.zeros((m, m, n))
    f2 = np.zeros((m, n, n))
    for i in range(m):
        for j in range(n):
            for k in range(m):
                for l in range(n):
                    f1[i, k, j] += pi[i, j, k, l]
                    f2[k, j, l] += pi[i, j, k, l]
    return f1, f2


def _pack(f1, f2, m, n):
    x = np.zeros(m * m * n + m * n * n)
    for i in range(m):
        for k in range(m):
            for j in range(n):
                x[rm.f1_index(i, k, j, m, n)] = f1[i, k, j]
    for k in range(m):
        for j in range(n):
            for l in range(n):
                x[rm.f2_index(k, j, l, m, n)] = f2[k, j, l]
    return x


@pytest.mark.parametrize("m,n", [(2, 3), (3, 3), (4, 2)])
def test_constraints_and_cost_mean_what_eq3_says(m, n):
    """Any transport plan of eq. (1) routed through (k, j) gives flows with
    A x = b and <c, x> = sum c_{ij;kl} pi_{ij;kl} (separable cost, eq. 2-3).
    This ties the vec order of A, b, c to the meaning of f1, f2, mu1, mu2."""
    rng = np.random.default_rng(7)
    pi = rng.random((m, n, m, n))
    pi /= pi.sum()
    mu1 = pi.sum(axis=(2, 3))
    mu2 = pi.sum(axis=(0, 1))
    f1, f2 = _flows_from_plan(pi, m, n)
    x = _pack(f1, f2, m, n)
    A = rm.build_A(m, n)
    np.testing.assert_allclose(A @ x, rm.build_b(mu1, mu2), atol=1e-14)
    np.testing.assert_allclose(rm.build_A_hat(m, n) @ x, rm.build_b_hat(mu1, mu2), atol=1e-14)
    c = rm.build_c(m, n)
    direct = sum(pi[i, j, k, l] * ((i - k) ** 2 + (j - l) ** 2)
                 for i in range(m) for j in range(n) for k in range(m) for l in range(n))
    assert abs(c @ x - direct) < 1e-13
    f1b, f2b = rm.split_x(x, m, n)
    np.testing.assert_array_equal(f1b, f1)
    np.testing.assert_array_equal(f2b, f2)


def test_cost_entries():
    m, n = 4, 3
    c = rm.build_c(m, n)
    for i in range(m):
        for k in range(m):
            for j in range(n):
                assert c[rm.f1_index(i, k, j, m, n)] == (k - i) ** 2
    for k in range(m):
        for j in range(n):
            for l in range(n):
                assert c[rm.f2_index(k, j, l, m, n)] == (j - l) ** 2


def test_vec_is_column_major():
    mu = np.arange(6.0).reshape(2, 3)          # mu[i, j]
    v = rm.vec(mu)
    for i in range(2):
        for j in range(3):
            assert v[i + 2 * j] == mu[i, j]
    np.testing.assert_array_equal(rm.unvec(v, 2, 3), mu)
