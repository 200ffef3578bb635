"""Pins of the oracle's Algorithm 2 (HOT) against the paper's own statements,
closed forms and exact LP values."""
import json
import math
import os

import numpy as np
import pytest

from oracle import hot, exact, closed_forms
from oracle import reduced_model as rm
from paper_2408_00598_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_ot_cases.json")


def lagrangian(A, b, c, sigma, y, z, x):
    """L_sigma(y, z; x) exactly as printed in Sec. III-A (z >= 0 assumed)."""
    r = A.T @ y + z - c + x / sigma
    return -b @ y + 0.5 * sigma * (r @ r) - (x @ x) / sigma


def _random_state(m, n, seed):
    rng = np.random.default_rng(seed)
    mu1, mu2 = syn.make_pair("white", m, seed, n)
    A = rm.build_A(m, n)
    b = rm.build_b(mu1, mu2)
    c = rm.build_c(m, n) / hot.cost_scale(rm.build_c(m, n))
    N = c.size
    x = rng.standard_normal(N) * 0.01
    z = np.abs(rng.standard_normal(N))
    return A, b, c, x, z


def step_invariants(A, b, c, sigma, x, z, y_bar, x_bar, z_bar):
    """Facts the paper proves about one step (App. C): A x-bar = b, and
    x~ = x-bar + sigma(A^T y-bar + z-bar - c) is >= 0 and orthogonal to z-bar."""
    primal = np.abs(A @ x_bar - b).max()
    xt = x_bar + sigma * (A.T @ y_bar + z_bar - c)
    return primal, -min(0.0, xt.min()), abs(xt @ z_bar), z_bar.min()


@pytest.mark.parametrize("m,n,seed", [(3, 3, 1), (4, 5, 2), (5, 3, 3)])
def test_step1_minimises_the_augmented_lagrangian(m, n, seed):
    A, b, c, x, z = _random_state(m, n, seed)
    sigma = 0.37
    y_bar, x_bar, z_bar = hot.hot_step(A, b, c, sigma, x, z, m, n)
    L0 = lagrangian(A, b, c, sigma, y_bar, z, x)
    rng = np.random.default_rng(0)
    # gradient by central differences of the printed L_sigma vanishes at y-bar
    h = 1e-5
    for q in rng.choice(y_bar.size, 6, replace=False):
        e = np.zeros_like(y_bar)
        e[q] = h
        g = (lagrangian(A, b, c, sigma, y_bar + e, z, x) - lagrangian(A, b, c, sigma, y_bar - e, z, x)) / (2 * h)
        assert abs(g) < 1e-6
    for _ in range(5):
        d = rng.standard_normal(y_bar.size) * 1e-2
        assert lagrangian(A, b, c, sigma, y_bar + d, z, x) >= L0 - 1e-12


@pytest.mark.parametrize("m,n,seed", [(3, 3, 4), (4, 5, 5)])
def test_step3_minimises_over_the_cone(m, n, seed):
    A, b, c, x, z = _random_state(m, n, seed)
    sigma = 1.3
    y_bar, x_bar, z_bar = hot.hot_step(A, b, c, sigma, x, z, m, n)
    assert z_bar.min() >= 0.0
    L0 = lagrangian(A, b, c, sigma, y_bar, z_bar, x_bar)
    rng = np.random.default_rng(1)
    for _ in range(20):
        zz = np.maximum(z_bar + rng.standard_normal(z_bar.size) * 1e-2, 0.0)
        assert lagrangian(A, b, c, sigma, y_bar, zz, x_bar) >= L0 - 1e-12


@pytest.mark.parametrize("m,n,seed", [(3, 3, 6), (4, 5, 7), (6, 6, 8)])
def test_step_invariants(m, n, seed):
    A, b, c, x, z = _random_state(m, n, seed)
    sigma = 0.05
    out = hot.hot_step(A, b, c, sigma, x, z, m, n)
    primal, neg, orth, zmin = step_invariants(A, b, c, sigma, x, z, *out)
    assert primal < 1e-13
    assert neg < 1e-14
    assert orth < 1e-13
    assert zmin >= 0.0


def test_min_equals_projection_form():
    """z - Pi_+(z - x) = min(x, z): the two forms of the middle KKT term
    (Sec. III-A mapping and eq. kkt_res) agree."""
    rng = np.random.default_rng(3)
    x, z = rng.standard_normal(1000), rng.standard_normal(1000)
    np.testing.assert_allclose(z - np.maximum(z - x, 0.0), np.minimum(x, z), atol=0)


def test_rate_bound_of_the_unrestarted_iteration():
    """Prop. 3 (Sec. III-A): ||R(w-bar^k)|| <= (sigma+1)/sigma * R0/(k+1) for
    Algorithm 2 as printed (fixed anchor w^0 = 0, fixed sigma), R0 measured to a
    KKT point (x*, z*) (the bound holds for any fixed point of the operator)."""
    m = n = 6
    mu1, mu2 = syn.make_pair("gauss", m, 11)
    A = rm.build_A(m, n)
    b = rm.build_b(mu1, mu2)
    c = rm.build_c(m, n) / hot.cost_scale(rm.build_c(m, n))
    ref = hot.hot_solve(mu1, mu2, tol=1e-12, max_iter=200000)
    scale = ref.cost_scale
    x_star, z_star = ref.x, ref.z / scale
    sigma = 0.05
    R0 = np.linalg.norm(x_star + sigma * z_star)
    worst = []

    def on_iterate(total, sig, x, z, x_bar, y_bar, z_bar):
        R = hot.kkt_mapping(A, b, c, x_bar, y_bar, z_bar)
        nrm = math.sqrt(sum(float(v @ v) for v in R))
        k = total - 1
        worst.append(nrm * (k + 1) / ((sigma + 1) / sigma * R0))

    p = hot.HotParams(sigma0=sigma, restart=False, check_every=1)
    hot.hot_solve(mu1, mu2, tol=0.0, max_iter=400, params=p, on_iterate=on_iterate)
    assert len(worst) == 400
    assert max(worst) <= 1.0 + 1e-6


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hot_reaches_hand_derived_values(case):
    mu1 = np.array(case["mu1"], dtype=float)
    mu2 = np.array(case["mu2"], dtype=float)
    r = hot.hot_solve(mu1, mu2, tol=1e-10, max_iter=200000)
    assert r.converged
    assert abs(r.ot_value - case["value"]) <= 1e-6 * max(1.0, case["value"])


@pytest.mark.parametrize("kind,S,seed", [("white", 8, 1), ("gauss", 8, 2), ("shapes", 8, 3),
                                         ("cauchy", 10, 4), ("white", 12, 5)])
def test_hot_matches_exact_min_cost_flow(kind, S, seed):
    mu1, mu2 = syn.make_pair(kind, S, seed)
    ex = exact.ot_exact_mcf(mu1, mu2)
    r = hot.hot_solve(mu1, mu2, tol=1e-10, max_iter=200000)
    assert r.converged and r.rel_kkt <= 1e-10
    assert abs(r.ot_value - ex) <= 2e-7 * ex
    assert abs(r.dual_value - ex) <= 2e-7 * ex
    # the reported iterate satisfies the paper's quality measures (Sec. IV-A)
    A = rm.build_A(S, S)
    assert hot.feaserr(A, rm.build_b(mu1, mu2), r.x) <= 1e-8


def test_translation_closed_form():
    mu1, mu2, s, t = syn.make_translation(12, 21)
    r = hot.hot_solve(mu1, mu2, tol=1e-10, max_iter=200000)
    assert abs(r.ot_value - closed_forms.translation_value(s, t)) <= 1e-6 * (s * s + t * t)


def test_product_measure_closed_form():
    rng = np.random.default_rng(5)
    p, q, p2, q2 = (rng.random(10) for _ in range(4))
    p, q, p2, q2 = (v / v.sum() for v in (p, q, p2, q2))
    mu1, mu2 = np.outer(p, q), np.outer(p2, q2)
    r = hot.hot_solve(mu1, mu2, tol=1e-10, max_iter=200000)
    ref = closed_forms.product_measure_value(p, q, p2, q2)
    assert abs(r.ot_value - ref) <= 1e-6 * ref


def test_rectangular_grid_and_coordinates():
    """m != n and non-uniform coordinates (Sec. IV-B / App. E bins) against the exact LP."""
    rng = np.random.default_rng(9)
    m, n = 5, 7
    mu1, mu2 = syn.make_pair("gauss", m, 3, n)
    xs = np.cumsum(rng.uniform(0.5, 2.0, m))
    ys = np.cumsum(rng.uniform(0.5, 2.0, n))
    ex = exact.ot_exact_lp(mu1, mu2, xs, ys)
    r = hot.hot_solve(mu1, mu2, tol=1e-10, max_iter=200000, xs=xs, ys=ys)
    assert abs(r.ot_value - ex) <= 1e-6 * ex


def test_iteration_cap_and_trace():
    mu1, mu2 = syn.make_pair("white", 6, 2)
    r = hot.hot_solve(mu1, mu2, tol=1e-14, max_iter=35)
    assert not r.converged
    assert r.iters == 40                      # first check iteration at or past the cap
    assert [t[0] for t in r.trace] == [10, 20, 30, 40]
