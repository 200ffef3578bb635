"""Rectangular grids, m != n (eq. 1 on an m x n grid).  The slab layout then
holds n f1 slabs of m x m and m f2 slabs of n x n, Prop. 3 runs with its
general m and n, and Algorithm 1 couples m sources with n sinks per node.
Checked against the FP64 oracle (iterates in FP64 mode, values at the
paper's stopping rule in FP32 mode), the exact LP, and the oracle's
Algorithm 1 run on the GPU's own flows."""
import numpy as np
import pytest

from oracle import exact
from oracle import hot as ohot
from oracle import recover as orec
from oracle import reduced_model as rm
from paper_2408_00598_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hot():
    from paper_2408_00598_gb300 import hot
    hot.load_library()
    return hot


@pytest.mark.parametrize("m,n,kind", [(8, 12, "gauss"), (20, 8, "white"), (12, 36, "shapes")])
@pytest.mark.parametrize("iters", [10, 80])
def test_fp64_iterates_match_oracle(hot, m, n, kind, iters):
    mu1, mu2 = syn.make_pair(kind, m, 7, n=n)
    ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=iters)
    with hot.Context(precision="fp64") as ctx:
        r = ctx.solve(mu1, mu2, tol=0.0, max_iter=iters)
        x = ctx.flows(r)
        ctx.release(r)
    assert (r["m"], r["n"]) == (m, n)
    assert r["iters"] == ref.iters and r["restarts"] == ref.restarts
    assert r["cost_scale"] == ref.cost_scale
    assert np.abs(x - ref.x).max() <= 1e-10 * np.abs(ref.x).max()
    assert abs(r["rel_kkt"] - ref.rel_kkt) <= 1e-6 * ref.rel_kkt


@pytest.mark.parametrize("m,n,kind,seed", [(16, 40, "white", 1), (44, 24, "shapes", 2), (40, 20, "cauchy", 3), (32, 64, "white", 3)])
def test_fp32_value_parity_at_paper_stopping_rule(hot, m, n, kind, seed):
    """Relative KKT 1e-6 (eq. kkt_res): FP32 bulk value within 1e-6 of the oracle."""
    mu1, mu2 = syn.make_pair(kind, m, seed, n=n)
    ref = ohot.hot_solve(mu1, mu2, tol=1e-6, max_iter=100000)
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-6, max_iter=100000)
        ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-6
    assert abs(r["ot_value"] - ref.ot_value) <= 1e-6 * abs(ref.ot_value), (r["iters"], ref.iters)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_value_against_exact_lp(hot, precision):
    m, n = 12, 20
    mu1, mu2 = syn.make_pair("gauss", m, 5, n=n)
    ex = exact.ot_exact_lp(mu1, mu2)
    with hot.Context(precision=precision) as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-8, max_iter=300000)
        ctx.release(r)
    assert r["status"] == 0
    assert abs(r["dual_value"] - ex) <= 1e-6 * ex
    assert abs(r["ot_value"] - ex) <= 1e-5 * ex


def test_coordinates_on_a_rectangular_grid(hot):
    """Non-uniform bin positions along both axes (FP64 mode), iterates as the oracle's."""
    m, n = 12, 24
    mu1, mu2 = syn.make_pair("cauchy", m, 4, n=n)
    rng = np.random.default_rng(4)
    xs = np.cumsum(rng.uniform(0.3, 2.0, m))
    ys = np.cumsum(rng.uniform(0.3, 2.0, n)) - 5.0
    ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=60, xs=xs, ys=ys)
    with hot.Context(precision="fp64") as ctx:
        r = ctx.solve(mu1, mu2, tol=0.0, max_iter=60, xs=xs, ys=ys)
        x = ctx.flows(r)
        ctx.release(r)
    assert r["iters"] == ref.iters and r["restarts"] == ref.restarts
    assert np.abs(x - ref.x).max() <= 1e-10 * np.abs(ref.x).max()


@pytest.mark.parametrize("precision,m,n", [("fp64", 12, 20), ("fp32", 36, 16), ("fp32", 24, 72)])
def test_recovery_matches_oracle_algorithm1_on_the_same_flows(hot, precision, m, n):
    """Algorithm 1 on the GPU vs the oracle's literal loops on the GPU's own
    x-bar: the same entries (FP64 pairs of the FP32 flows hold their prefix
    sums to about 48 bits, so masses agree to 1e-12 of the total)."""
    mu1, mu2 = syn.make_pair("white", m, 9, n=n)
    with hot.Context(precision=precision) as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-7, max_iter=200000)
        x = ctx.flows(r)
        src, dst, mass, l1 = ctx.recover_plan(r)
        ctx.release(r)
    ent = orec.recover_from_x(x, m, n)
    Po = np.zeros((m * n, m * n))
    for i, j, k, l, p in ent:
        Po[i * n + j, k * n + l] += p
    Pg = np.zeros((m * n, m * n))
    np.add.at(Pg, (src, dst), mass)
    assert np.abs(Pg - Po).max() <= (1e-14 if precision == "fp64" else 1e-12)
    assert mass.min() > 0
    # ordered by node (k, j), at most m + n - 1 entries per node
    node = (dst // n) * n + (src % n)
    assert np.all(np.diff(node) >= 0)
    assert np.bincount(node).max() <= m + n - 1
    rs, ts = orec.plan_marginals(ent, m, n)
    assert abs(l1[0] - np.abs(rs - mu1).sum()) <= 1e-10
    assert abs(l1[1] - np.abs(ts - mu2).sum()) <= 1e-10
    # the plan's cost is at most the cost of the clipped flows (App. C)
    cost = (((src // n) - (dst // n)) ** 2 + ((src % n) - (dst % n)) ** 2) @ mass
    assert cost <= rm.build_c(m, n) @ np.maximum(x, 0.0) * (1 + 1e-9)


def test_batch_mixes_shapes(hot):
    """One batch of square and rectangular pairs solves each as alone."""
    shapes = [(16, 16), (8, 28), (24, 12), (20, 20)]
    pairs = [syn.make_pair("white", m, 11 + q, n=n) for q, (m, n) in enumerate(shapes)]
    with hot.Context(precision="fp32") as ctx:
        single = []
        for a, b in pairs:
            r = ctx.solve(a, b, tol=1e-6)
            ctx.release(r)
            single.append(r)
        batch = ctx.solve_batch([a for a, _ in pairs], [b for _, b in pairs], tol=1e-6)
    for s, b in zip(single, batch):
        assert (b["m"], b["n"]) == (s["m"], s["n"])
        assert b["iters"] == s["iters"] and b["ot_value"] == s["ot_value"]
