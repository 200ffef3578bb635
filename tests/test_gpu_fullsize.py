"""Full-size cases (256 x 256 and 512 x 512, 3.4e7 and 2.7e8 flow variables),
checked by properties that hold at any size: textbook closed forms of the
optimal value (integer translation, product measures), the stopping rule, and
the marginals of the recovered plan.

At the paper's stopping rule (relative KKT 1e-6 in 2-norms over 1e7..1e8
entries) neither objective is close to the optimum on these grids: measured
on the pairs below, the dual <b, y-bar> is within 0.4..1.3 % and the primal
<c, x-bar> can be far off, because the rule tolerates a negative part of
x-bar of L1 size up to about sigma sqrt(V) ||A^T y + z - c||.  At relative
KKT 1e-8 the dual is within 2e-7..5e-5 of the closed form.  The closed forms
are therefore checked on the dual objective at 1e-8 (and loosely at 1e-6)."""
import numpy as np
import pytest

from oracle import closed_forms
from paper_2408_00598_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(precision="fp32")
    yield c
    c.close()


@pytest.fixture(scope="module")
def lib():
    from paper_2408_00598_gb300 import hot
    hot.load_library()
    return hot


def test_translation_256(ctx):
    mu1, mu2, s, t = syn.make_translation(256, 3, base_kind="gauss")
    exact = closed_forms.translation_value(s, t)
    r = ctx.solve(mu1, mu2, tol=1e-6, max_iter=300000)
    n, l1 = ctx.recover_plan(r, device_out=())
    ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-6
    assert abs(r["dual_value"] - exact) <= 5e-2 * exact
    assert n <= 256 * 256 * (2 * 256 - 1)
    r = ctx.solve(mu1, mu2, tol=1e-8, max_iter=300000)
    ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-8
    assert abs(r["dual_value"] - exact) <= 2e-5 * exact


def test_product_measure_256(ctx):
    rng = np.random.default_rng(4)
    p, q, p2, q2 = (rng.uniform(0.1, 1.0, 256) for _ in range(4))
    p, q, p2, q2 = (v / v.sum() for v in (p, q, p2, q2))
    exact = closed_forms.product_measure_value(p, q, p2, q2)
    r = ctx.solve(np.outer(p, q), np.outer(p2, q2), tol=1e-8, max_iter=300000)
    ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-8
    assert abs(r["dual_value"] - exact) <= 2e-5 * exact
    assert abs(r["ot_value"] - exact) <= 1e-3 * exact


def test_white_noise_256_gap_and_plan(lib, ctx):
    import torch
    mu1, mu2 = syn.make_pair("white", 256, 1)
    r = ctx.solve(mu1, mu2, tol=1e-6, max_iter=200000)
    n, l1 = ctx.recover_plan(r, device_out=())
    src = torch.empty(n, dtype=torch.int32, device="cuda")
    dst = torch.empty(n, dtype=torch.int32, device="cuda")
    mass = torch.empty(n, dtype=torch.float64, device="cuda")
    n2, _ = ctx.recover_plan(r, device_out=(src, dst, mass))
    ctx.release(r)
    assert n2 == n
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-6
    S = 256
    m1 = torch.zeros(S * S, dtype=torch.float64, device="cuda").index_add_(0, src.long(), mass)
    assert abs(torch.abs(m1.cpu() - torch.from_numpy(mu1.reshape(-1))).sum().item() - l1[0]) <= 1e-9
    assert (mass > 0).all().item()
    node = (dst.long() // S) * S + (src.long() % S)
    assert (node[1:] >= node[:-1]).all().item()
    assert torch.bincount(node).max().item() <= 2 * S - 1


def test_translation_512(ctx):
    """512 x 512 (2.7e8 flow variables, about 2.7 GB of FP32 state)."""
    mu1, mu2, s, t = syn.make_translation(512, 5, base_kind="shapes")
    exact = closed_forms.translation_value(s, t)
    r = ctx.solve(mu1, mu2, tol=1e-8, max_iter=300000)
    ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 1e-8
    assert abs(r["dual_value"] - exact) <= 2e-4 * exact


# ------------------------------------------- the 256 x 256 benchmark pair --

def test_benchmark_pair_plan_marginals_and_algorithm1(ctx):
    """The throughput benchmark's 256 x 256 white-noise pair (seed 1000) solved
    to relative KKT 5e-10: the recovered plan's marginals agree with mu and nu
    to 1e-6 in L1 (recomputed here on the host from the returned entries), and
    Algorithm 1 on the device gives, node by node, the entries of the oracle's
    literal loops (Alg. 1) run on the same clipped flows, for 64 sampled nodes
    (k, j)."""
    from oracle import recover as orec
    from oracle import reduced_model as rm
    S = 256
    mu1, mu2 = syn.make_pair("white", S, 1000)
    # measured on this pair: relative KKT 1e-8 (37,800 iterations) leaves
    # 3.6e-6 in L1, 1e-9 (57,070) 1.4e-6, 5e-10 (69,720) 3.3e-7
    r = ctx.solve(mu1, mu2, tol=5e-10, max_iter=1000000)
    x = ctx.flows(r)
    src, dst, mass, l1 = ctx.recover_plan(r)
    ctx.release(r)
    assert r["status"] == 0 and r["rel_kkt"] <= 5e-10
    m1 = np.bincount(src, weights=mass, minlength=S * S).reshape(S, S)
    m2 = np.bincount(dst, weights=mass, minlength=S * S).reshape(S, S)
    e1, e2 = np.abs(m1 - mu1).sum(), np.abs(m2 - mu2).sum()
    assert e1 <= 1e-6 and e2 <= 1e-6, (e1, e2)
    assert abs(e1 - l1[0]) <= 1e-9 and abs(e2 - l1[1]) <= 1e-9
    assert mass.min() > 0
    node = (dst.astype(np.int64) // S) * S + (src % S)
    assert np.all(np.diff(node) >= 0)
    f1, f2 = rm.split_x(x, S, S)
    rng = np.random.default_rng(7)
    picks = rng.choice(S * S, 64, replace=False)
    lo = np.searchsorted(node, picks, side="left")
    hi = np.searchsorted(node, picks, side="right")
    worst = 0.0
    for q, nd in enumerate(picks):
        k, j = divmod(int(nd), S)
        ref = orec.recover_cell(np.maximum(f1[:, k, j], 0.0), np.maximum(f2[k, j, :], 0.0))
        want = {(i, l): p for i, l, p in ref}
        got = {}
        for e in range(lo[q], hi[q]):
            got[(int(src[e]) // S, int(dst[e]) % S)] = float(mass[e])
        for key in set(want) | set(got):
            worst = max(worst, abs(want.get(key, 0.0) - got.get(key, 0.0)))
    # FP64 pairs of the FP32 flows hold the prefix sums to about 48 bits
    assert worst <= 1e-12, worst
