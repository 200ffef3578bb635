"""Pins of Algorithm 1 (plan recovery), the exact solvers and the closed forms."""
import json
import os

import numpy as np
import pytest

from oracle import exact, closed_forms, recover
from oracle import reduced_model as rm
from paper_2408_00598_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_ot_cases.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_exact_solvers_on_hand_derived_cases(case):
    mu1 = np.array(case["mu1"], dtype=float)
    mu2 = np.array(case["mu2"], dtype=float)
    v = case["value"]
    assert abs(exact.ot_exact_mcf(mu1, mu2) - v) <= 1e-12 * max(1, v)
    assert abs(exact.ot_exact_lp(mu1, mu2) - v) <= 1e-9 * max(1, v)
    assert abs(exact.reduced_exact_lp(mu1, mu2) - v) <= 1e-9 * max(1, v)


@pytest.mark.parametrize("kind,S,seed", [("white", 4, 1), ("gauss", 6, 2), ("shapes", 6, 3),
                                         ("cauchy", 5, 4), ("white", 8, 5)])
def test_mcf_lp_and_reduced_model_agree(kind, S, seed):
    """Min-cost flow = LP of eq. (1) = LP of the reduced model eq. (3)
    (the equivalence the paper takes from Auricchio et al.)."""
    mu1, mu2 = syn.make_pair(kind, S, seed)
    a = exact.ot_exact_mcf(mu1, mu2)
    b = exact.ot_exact_lp(mu1, mu2)
    c = exact.reduced_exact_lp(mu1, mu2)
    assert abs(a - b) <= 1e-9 * max(1, b)
    assert abs(c - b) <= 1e-9 * max(1, b)


def test_mcf_brute_force_permutations():
    rng = np.random.default_rng(3)
    S = 5
    for trial in range(4):
        k = 5
        src = rng.choice(S * S, k, replace=False)
        dst = rng.choice(S * S, k, replace=False)
        mu1 = np.zeros((S, S))
        mu2 = np.zeros((S, S))
        for q in src:
            mu1[q // S, q % S] = 1.0 / k
        for q in dst:
            mu2[q // S, q % S] = 1.0 / k
        sb = [(q // S, q % S) for q in src]
        db = [(q // S, q % S) for q in dst]
        ref = closed_forms.brute_force_uniform(sb, db)
        assert abs(exact.ot_exact_mcf(mu1, mu2) - ref) <= 1e-12 * max(1, ref)


def test_mcf_product_measure_and_translation():
    rng = np.random.default_rng(4)
    p, q, p2, q2 = (rng.random(7) for _ in range(4))
    p, q, p2, q2 = (v / v.sum() for v in (p, q, p2, q2))
    ref = closed_forms.product_measure_value(p, q, p2, q2)
    assert abs(exact.ot_exact_mcf(np.outer(p, q), np.outer(p2, q2)) - ref) <= 1e-12
    for seed in range(3):
        mu1, mu2, s, t = syn.make_translation(10, seed)
        assert abs(exact.ot_exact_mcf(mu1, mu2) - (s * s + t * t)) <= 1e-9


def test_ot_1d_closed_form_matches_lp():
    """1D quantile formula against the LP on an m x 1 grid."""
    rng = np.random.default_rng(8)
    p, p2 = rng.random(9), rng.random(9)
    p, p2 = p / p.sum(), p2 / p2.sum()
    ref = exact.ot_exact_lp(p[:, None], p2[:, None])
    assert abs(closed_forms.ot_1d(p, p2) - ref) <= 1e-10


@pytest.mark.parametrize("kind,S,seed", [("white", 5, 1), ("gauss", 6, 2), ("shapes", 7, 3)])
def test_algorithm1_on_an_exact_reduced_optimum(kind, S, seed):
    """Prop. 1: on an optimal (f1, f2), Algorithm 1 returns a feasible plan of
    eq. (1) whose cost is the optimal value; north-west-corner coupling per
    node has at most m + n - 1 nonzeros."""
    mu1, mu2 = syn.make_pair(kind, S, seed)
    val, x = exact.reduced_exact_lp(mu1, mu2, want_x=True)
    ent = recover.recover_from_x(x, S, S)
    r, s = recover.plan_marginals(ent, S, S)
    assert np.abs(r - mu1).sum() <= 1e-9
    assert np.abs(s - mu2).sum() <= 1e-9
    assert abs(recover.plan_cost(ent) - exact.ot_exact_mcf(mu1, mu2)) <= 1e-9
    per_node = {}
    for i, j, k, l, p in ent:
        per_node[(k, j)] = per_node.get((k, j), 0) + 1
        assert p > 0
    assert max(per_node.values()) <= 2 * S - 1


def test_algorithm1_cell_by_hand():
    """One node: a = (0.5, 0.3, 0.2), b = (0.4, 0.6) -> north-west corner:
    (0,0) 0.4, (0,1) 0.1, (1,1) 0.3, (2,1) 0.2."""
    out = recover.recover_cell([0.5, 0.3, 0.2], [0.4, 0.6])
    got = [(i, l, round(p, 12)) for i, l, p in out]
    assert got == [(0, 0, 0.4), (0, 1, 0.1), (1, 1, 0.3), (2, 1, 0.2)]


def test_algorithm1_leftover_when_node_is_unbalanced():
    """Reading for approximate flows: mass a node cannot pass on stays unassigned."""
    out = recover.recover_cell([0.5, 0.5], [0.3, 0.3])
    assert abs(sum(p for _, _, p in out) - 0.6) < 1e-15
