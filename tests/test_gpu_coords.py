"""Bins with given coordinates (hot_solve_coords): the cost of moving mass from
bin (i, j) to (k, l) is (xs_i - xs_k)^2 + (ys_j - ys_l)^2 (eq. 1 with the
bins' own positions, as colour and point-cloud data have).  Checked against
the FP64 oracle run on the same coordinates (iterates in FP64 mode, values in
FP32 mode with integer and with real-valued coordinates) and against the
exact LP."""
import numpy as np
import pytest

from oracle import exact
from oracle import hot as ohot
from paper_2408_00598_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hot():
    from paper_2408_00598_gb300 import hot
    hot.load_library()
    return hot


def _coords(S, seed, integer):
    rng = np.random.default_rng(seed)
    step = rng.integers(1, 4, size=(2, S)) if integer else rng.uniform(0.3, 2.0, size=(2, S))
    xs = np.cumsum(step[0]).astype(float) - 3.0
    ys = np.cumsum(step[1]).astype(float)
    return xs, ys


@pytest.mark.parametrize("S,kind,seed", [(12, "gauss", 1), (16, "white", 2)])
@pytest.mark.parametrize("iters", [10, 80])
def test_fp64_iterates_match_oracle(hot, S, kind, seed, iters):
    mu1, mu2 = syn.make_pair(kind, S, seed)
    xs, ys = _coords(S, seed, integer=False)
    ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=iters, xs=xs, ys=ys)
    with hot.Context(precision="fp64") as ctx:
        r = ctx.solve(mu1, mu2, tol=0.0, max_iter=iters, xs=xs, ys=ys)
        x = ctx.flows(r)
        ctx.release(r)
    assert r["iters"] == ref.iters and r["restarts"] == ref.restarts
    assert r["cost_scale"] == ref.cost_scale
    assert np.abs(x - ref.x).max() <= 1e-10 * np.abs(ref.x).max()


@pytest.mark.parametrize("precision,integer", [("fp64", False), ("fp32", True)])
def test_value_against_exact_lp(hot, precision, integer):
    S = 12
    mu1, mu2 = syn.make_pair("gauss", S, 5)
    xs, ys = _coords(S, 5, integer)
    ex = exact.ot_exact_lp(mu1, mu2, xs, ys)
    with hot.Context(precision=precision) as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-8, max_iter=300000, xs=xs, ys=ys)
        ctx.release(r)
    assert r["status"] == 0
    assert abs(r["dual_value"] - ex) <= 1e-6 * ex
    assert abs(r["ot_value"] - ex) <= 1e-5 * ex


@pytest.mark.parametrize("S,kind,seed", [(16, "shapes", 3), (24, "white", 4)])
def test_fp32_integer_coordinates_match_oracle(hot, S, kind, seed):
    """Same-rule parity at the paper's stopping rule, as for the unit grid."""
    mu1, mu2 = syn.make_pair(kind, S, seed)
    xs, ys = _coords(S, seed, integer=True)
    ref = ohot.hot_solve(mu1, mu2, tol=1e-6, max_iter=100000, xs=xs, ys=ys)
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-6, max_iter=100000, xs=xs, ys=ys)
        ctx.release(r)
    assert r["status"] == 0 and r["iters"] == ref.iters
    assert abs(r["ot_value"] - ref.ot_value) <= 1e-6 * abs(ref.ot_value)


def test_unit_coordinates_equal_the_plain_solve(hot):
    S = 16
    mu1, mu2 = syn.make_pair("cauchy", S, 6)
    grid = np.arange(S, dtype=float)
    with hot.Context(precision="fp32") as ctx:
        a = ctx.solve(mu1, mu2, tol=1e-6)
        b = ctx.solve(mu1, mu2, tol=1e-6, xs=grid, ys=grid)
        ctx.release(a)
        ctx.release(b)
    assert a["ot_value"] == b["ot_value"] and a["iters"] == b["iters"]


@pytest.mark.parametrize("m,n,kind,seed", [(16, 16, "white", 11), (24, 24, "gauss", 12), (13, 19, "shapes", 13)])
def test_fp32_real_coordinates_match_oracle(hot, m, n, kind, seed):
    """Real-valued bin positions (sorted U(0, 1), as colour or point-cloud bins
    have; App. E-G) in FP32 bulk mode: the reduced cost and the objective's
    parts are formed in pairs.  FP32 mode solves eq. (1) with the positions
    rounded to FP32, so the FP64 oracle runs on those rounded positions; at
    the paper's stopping rule: the dual to 1e-6, the primal to 1e-6 of
    sum |c x-bar|, iterations within a check or two."""
    from oracle import reduced_model as rm
    rng = np.random.default_rng(seed)
    xs, ys = np.sort(rng.uniform(0.0, 1.0, m)), np.sort(rng.uniform(0.0, 1.0, n))
    mu1, mu2 = syn.make_pair(kind, m, seed, n=n)
    r32 = lambda v: v.astype(np.float32).astype(np.float64)
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=1e-6, max_iter=100000, xs=xs, ys=ys)
        x = ctx.flows(r)
        ctx.release(r)
    xs, ys = r32(xs), r32(ys)
    ref = ohot.hot_solve(mu1, mu2, tol=1e-6, max_iter=100000, xs=xs, ys=ys)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-6
    assert abs(r["iters"] - ref.iters) <= max(20, 0.01 * ref.iters), (r["iters"], ref.iters)
    if r["iters"] != ref.iters:
        ref = ohot.hot_solve(mu1, mu2, tol=0.0, max_iter=r["iters"], xs=xs, ys=ys)
    assert abs(r["dual_value"] - ref.dual_value) <= 1e-6 * abs(ref.dual_value)
    cx = float(np.abs(rm.build_c(m, n, xs, ys) * x).sum())
    assert abs(r["ot_value"] - ref.ot_value) <= 1e-6 * max(cx, abs(ref.ot_value))


def test_fp32_real_coordinates_against_exact_lp(hot):
    """A tight stopping rule: both objectives at the exact optimum of eq. (1)
    with real-valued positions, rounded to FP32 as FP32 mode solves it."""
    S = 8
    rng = np.random.default_rng(21)
    xs, ys = np.sort(rng.uniform(0.0, 3.0, S)), np.sort(rng.uniform(0.0, 3.0, S))
    mu1, mu2 = syn.make_pair("white", S, 21)
    ex = exact.ot_exact_lp(mu1, mu2, xs.astype(np.float32).astype(np.float64),
                           ys.astype(np.float32).astype(np.float64))
    with hot.Context(precision="fp32") as ctx:
        r = ctx.solve(mu1, mu2, tol=5e-9, max_iter=400000, xs=xs, ys=ys)
        ctx.release(r)
    assert r["status"] == 0
    assert abs(r["dual_value"] - ex) <= 1e-6 * ex
    assert abs(r["ot_value"] - ex) <= 2e-6 * ex


def test_coordinates_must_be_finite(hot):
    S = 8
    mu1, mu2 = syn.make_pair("white", S, 1)
    with hot.Context(precision="fp32") as ctx:
        with pytest.raises(hot.HotError) as e:
            ctx.solve(mu1, mu2, xs=np.array([0.0] * (S - 1) + [np.inf]), ys=np.arange(S, dtype=float))
    assert e.value.status == hot.HOT_EINVAL
