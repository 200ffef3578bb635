"""Pins of the oracle's two variants of Algorithm 2: the generalized ADMM the
paper compares against (Sec. IV-A: Step 4 replaced by
w^{k+1} = (1 - rho) w^k + rho w-bar^k, rho = 1.7) and the absolute-KKT stopping
rule of Table VI (the terms of eq. (kkt_res) without normalisers)."""
import numpy as np
import pytest

from oracle import hot, exact
from oracle import reduced_model as rm
from paper_2408_00598_gb300 import synthetic as syn


def _absolute_kkt_by_loops(mu1, mu2, c, x, y, z):
    """The absolute residual written out from the constraint definitions of
    eq. (3) with plain loops (no A): rows (k,j), (i,j), (k,l), last dropped."""
    m, n = mu1.shape
    f1 = {}
    f2 = {}
    # vec order of eq. (6): f1 index i + m k + m^2 j, f2 index m^2 n + k + m j + m n l
    for j in range(n):
        for k in range(m):
            for i in range(m):
                f1[i, k, j] = i + m * k + m * m * j
    for l in range(n):
        for j in range(n):
            for k in range(m):
                f2[k, j, l] = m * m * n + k + m * j + m * n * l
    # primal residual
    r2 = 0.0
    for k in range(m):
        for j in range(n):
            s = sum(x[f1[i, k, j]] for i in range(m)) - sum(x[f2[k, j, l]] for l in range(n))
            r2 += s * s
    for i in range(m):
        for j in range(n):
            s = sum(x[f1[i, k, j]] for k in range(m)) - mu1[i, j]
            r2 += s * s
    for k in range(m):
        for l in range(n):
            if (k, l) == (m - 1, n - 1):
                continue
            s = sum(x[f2[k, j, l]] for j in range(n)) - mu2[k, l]
            r2 += s * s
    # dual residual: (A^T y)_e from the rows that contain e
    y1 = lambda k, j: y[k + m * j]
    y2 = lambda i, j: y[m * n + i + m * j]
    def y3(k, l):
        if (k, l) == (m - 1, n - 1):
            return 0.0
        return y[2 * m * n + k + m * l]
    d2 = 0.0
    for (i, k, j), e in f1.items():
        t = y1(k, j) + y2(i, j) + z[e] - c[e]
        d2 += t * t
    for (k, j, l), e in f2.items():
        t = -y1(k, j) + y3(k, l) + z[e] - c[e]
        d2 += t * t
    mn2 = sum(min(a, b) ** 2 for a, b in zip(x, z))
    return max(np.sqrt(d2), np.sqrt(mn2), np.sqrt(r2))


@pytest.mark.parametrize("m,n,seed", [(3, 3, 1), (3, 4, 2)])
def test_absolute_kkt_equals_brute_force(m, n, seed):
    rng = np.random.default_rng(seed)
    mu1, mu2 = syn.make_pair("white", m, seed, n)
    A = rm.build_A(m, n)
    b = rm.build_b(mu1, mu2)
    c = rm.build_c(m, n) / 8.0
    x = rng.standard_normal(c.size)
    z = np.abs(rng.standard_normal(c.size))
    y = rng.standard_normal(A.shape[0])
    ref = _absolute_kkt_by_loops(mu1, mu2, c, x, y, z)
    assert abs(hot.kkt_absolute(A, b, c, x, y, z) - ref) <= 1e-12 * ref


def test_absolute_stop_rule_stops_on_the_absolute_residual():
    mu1, mu2 = syn.make_pair("gauss", 8, 4)
    p = hot.HotParams(stop="absolute")
    r = hot.hot_solve(mu1, mu2, tol=1e-9, max_iter=200000, params=p)
    assert r.converged and r.abs_kkt <= 1e-9
    # the iteration is the same as under the relative rule: only the test differs
    rr = hot.hot_solve(mu1, mu2, tol=1e-30, max_iter=r.iters)
    assert rr.iters == r.iters and abs(rr.abs_kkt - r.abs_kkt) <= 1e-15


@pytest.mark.parametrize("kind,S,seed", [("white", 8, 1), ("shapes", 8, 3)])
def test_gadmm_reaches_the_exact_optimum(kind, S, seed):
    mu1, mu2 = syn.make_pair(kind, S, seed)
    ex = exact.ot_exact_mcf(mu1, mu2)
    p = hot.HotParams(method="gadmm", relax=1.7)
    r = hot.hot_solve(mu1, mu2, tol=1e-10, max_iter=400000, params=p)
    assert r.converged
    assert abs(r.ot_value - ex) <= 2e-7 * ex
    assert abs(r.dual_value - ex) <= 2e-7 * ex


def test_unit_relaxation_is_plain_admm_and_halpern_first_step():
    """rho = 1: w^{k+1} = w-bar^k (ADMM with unit step, Sec. III-A); from w^0 = 0
    the Halpern step k = 0 gives w^1 = w^0/2 + (2 w-bar^0 - w^0)/2 = w-bar^0 too."""
    mu1, mu2 = syn.make_pair("white", 5, 6)
    seen = {}

    def record(tag):
        def cb(total, sigma, x, z, x_bar, y_bar, z_bar):
            seen.setdefault(tag, []).append((x.copy(), z.copy(), x_bar.copy(), z_bar.copy()))
        return cb

    noreset = dict(restart=False)
    hot.hot_solve(mu1, mu2, tol=0.0, max_iter=3, params=hot.HotParams(method="gadmm", relax=1.0, **noreset),
                  on_iterate=record("admm"))
    hot.hot_solve(mu1, mu2, tol=0.0, max_iter=3, params=hot.HotParams(**noreset), on_iterate=record("hot"))
    a, h = seen["admm"], seen["hot"]
    for k in range(len(a) - 1):               # ADMM: next iterate is this step's bar point
        np.testing.assert_array_equal(a[k + 1][0], a[k][2])
        np.testing.assert_array_equal(a[k + 1][1], a[k][3])
    np.testing.assert_allclose(h[1][0], a[1][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(h[1][1], a[1][1], rtol=0, atol=1e-15)


def test_relaxation_step_is_the_printed_combination():
    """One G-ADMM step moves w by rho (w-bar - w), rho = 1.7."""
    mu1, mu2 = syn.make_pair("gauss", 4, 7)
    seen = []
    hot.hot_solve(mu1, mu2, tol=0.0, max_iter=3,
                  params=hot.HotParams(method="gadmm", relax=1.7, restart=False),
                  on_iterate=lambda t, s, x, z, xb, yb, zb: seen.append((x.copy(), z.copy(), xb.copy(), zb.copy())))
    for k in range(2):
        x, z, xb, zb = seen[k]
        np.testing.assert_allclose(seen[k + 1][0], x + 1.7 * (xb - x), rtol=0, atol=1e-14)
        np.testing.assert_allclose(seen[k + 1][1], z + 1.7 * (zb - z), rtol=0, atol=1e-14)


def test_halpern_needs_fewer_iterations_than_gadmm():
    """The paper's Table II finding on a synthetic pair: Halpern acceleration
    reaches the tolerance in fewer iterations than the generalized ADMM."""
    mu1, mu2 = syn.make_pair("gauss", 10, 11)
    h = hot.hot_solve(mu1, mu2, tol=1e-6, max_iter=100000)
    g = hot.hot_solve(mu1, mu2, tol=1e-6, max_iter=100000, params=hot.HotParams(method="gadmm"))
    assert h.converged and g.converged
    assert h.iters < g.iters
