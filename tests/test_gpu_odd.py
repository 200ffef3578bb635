"""Grid sides that are not multiples of 4, down to 2 (eq. (1)-(3) define the
problem on any m x n grid with m, n >= 2).  The device stores every slab row
at a pitch rounded up to a multiple of 4; the pad columns hold zeros and
enter no sum, so the iterates, the values and the plan must be those of the
oracle on the unpadded model.
"""
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


@pytest.mark.parametrize("m,n,kind", [(9, 13, "white"), (13, 9, "gauss"), (5, 7, "shapes"), (2, 3, "white"),
                                      (3, 2, "cauchy"), (2, 2, "white"), (17, 17, "gauss"), (65, 65, "white")])
def test_fp64_iterates_match_oracle(hot, m, n, kind):
    """FP64 mode runs the oracle's arithmetic: x-bar after a fixed number of
    iterations (tol 0) to 1e-10, the same restarts and sigma."""
    iters = 40 if m * n > 1000 else 120
    mu1, mu2 = syn.make_pair(kind, m, 5, n=n)
    ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=iters)
    with hot.Context(precision="fp64") as ctx:
        r = ctx.solve(mu1, mu2, tol=0.0, max_iter=iters)
        x = ctx.flows(r)
        ctx.release(r)
    assert r["iters"] == ref.iters == iters
    assert r["restarts"] == ref.restarts
    assert abs(r["sigma"] - ref.sigma) <= 1e-9 * ref.sigma
    assert np.abs(x - ref.x).max() <= 1e-10 * np.abs(ref.x).max()
    assert abs(r["ot_value"] - ref.ot_value) <= 1e-10 * abs(ref.ot_value) + 1e-14


@pytest.mark.parametrize("m,n,kind", [(9, 13, "white"), (33, 17, "gauss"), (2, 3, "white"), (65, 65, "shapes")])
def test_fp32_iterates_track_oracle(hot, m, n, kind):
    iters = 60 if m * n > 1000 else 200
    mu1, mu2 = syn.make_pair(kind, m, 6, n=n)
    ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=iters)
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=0.0, max_iter=iters)
        x = ctx.flows(r)
        ctx.release(r)
    assert r["restarts"] == ref.restarts
    assert np.abs(x - ref.x).max() <= 1e-4 * np.abs(ref.x).max()
    assert abs(r["ot_value"] - ref.ot_value) <= 1e-5 * np.abs(rm.build_c(m, n) * ref.x).sum()


@pytest.mark.parametrize("m,n,kind", [(9, 13, "white"), (23, 11, "gauss"), (33, 45, "shapes")])
def test_fp32_value_parity_at_paper_stopping_rule(hot, m, n, kind):
    """Relative KKT 1e-6 (eq. kkt_res): FP32 bulk against the oracle, as in
    the parity test of the square grids (dual to 1e-6; primal to 1e-6 of
    sum |c x-bar|; the same iterate where the stop lands one check apart)."""
    mu1, mu2 = syn.make_pair(kind, m, 7, n=n)
    ref = ohot.hot_solve(mu1, mu2, tol=1e-6, max_iter=100000)
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-6, max_iter=100000)
        x = ctx.flows(r)
        ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-6
    assert abs(r["iters"] - ref.iters) <= max(20, 0.01 * ref.iters), (r["iters"], ref.iters)
    if r["iters"] != ref.iters:
        ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=r["iters"])
    assert abs(r["dual_value"] - ref.dual_value) <= 1e-6 * abs(ref.dual_value)
    cx = float(np.abs(rm.build_c(m, n) * x).sum())
    assert abs(r["ot_value"] - ref.ot_value) <= 1e-6 * max(cx, abs(ref.ot_value))


@pytest.mark.parametrize("m,n", [(5, 7), (7, 3), (6, 6)])
def test_values_against_the_exact_lp(hot, m, n):
    """FP64 at relative KKT 1e-10: the exact min-cost-flow optimum of eq. (1)."""
    mu1, mu2 = syn.make_pair("white", m, 8, n=n)
    ex = exact.ot_exact_mcf(mu1, mu2)
    with hot.Context(precision="fp64") as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-10, max_iter=400000)
        ctx.release(r)
    assert r["status"] == 0
    assert abs(r["ot_value"] - ex) <= 1e-6 * ex
    assert abs(r["dual_value"] - ex) <= 1e-6 * ex


@pytest.mark.parametrize("precision,m,n", [("fp64", 11, 7), ("fp32", 7, 11), ("fp32", 13, 13)])
def test_recovery_matches_oracle_algorithm1_on_the_same_flows(hot, precision, m, n):
    """Algorithm 1 on the device vs the oracle's literal loops on the device's
    own x-bar (the exported flows are unpadded, in the paper's vec order)."""
    mu1, mu2 = syn.make_pair("white", m, 9, n=n)
    with hot.Context(precision=precision) as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-7, max_iter=200000)
        x = ctx.flows(r)
        src, dst, mass, l1 = ctx.recover_plan(r)
        ctx.release(r)
    # the export is in the paper's order: A x-bar = b with the oracle's A
    A, b = rm.build_A(m, n), rm.build_b(mu1, mu2)
    assert np.abs(A @ x - b).max() <= 1e-6 * np.abs(b).max()
    ent = orec.recover_from_x(x, m, n)
    Po = np.zeros((m * n, m * n))
    for i, j, k, l, p in ent:
        Po[i * n + j, k * n + l] += p
    Pg = np.zeros((m * n, m * n))
    np.add.at(Pg, (src, dst), mass)
    assert np.abs(Pg - Po).max() <= (1e-14 if precision == "fp64" else 1e-12)
    rs, ts = orec.plan_marginals(ent, m, n)
    assert abs(l1[0] - np.abs(rs - mu1).sum()) <= 1e-10
    assert abs(l1[1] - np.abs(ts - mu2).sum()) <= 1e-10


def test_translation_65(hot):
    """An integer translation on a 65 x 65 grid: the value is the squared shift."""
    mu1, mu2, s, t = syn.make_translation(65, 3, base_kind="gauss")
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-9, max_iter=400000)
        ctx.release(r)
    ex = float(s * s + t * t)
    assert r["status"] == 0
    assert abs(r["dual_value"] - ex) <= 1e-5 * ex


def test_batch_of_odd_and_even_shapes_equals_single_solves(hot):
    shapes = [(9, 13), (16, 16), (5, 7), (65, 65), (2, 3)]
    pairs = [syn.make_pair("white", m, 11 + q, n=n) for q, (m, n) in enumerate(shapes)]
    with hot.Context(precision="fp32") as ctx:
        single = []
        for a, b in pairs:
            r = ctx.solve(a, b, tol=1e-6)
            ctx.release(r)
            single.append(r)
        batch = ctx.solve_batch([a for a, _ in pairs], [b for _, b in pairs], tol=1e-6)
    for s_, b_ in zip(single, batch):
        assert (b_["m"], b_["n"]) == (s_["m"], s_["n"])
        assert b_["iters"] == s_["iters"] and b_["ot_value"] == s_["ot_value"]
