"""Textbook closed forms that pin the oracle (test infrastructure only).

None of these is in the paper; they are standard facts about optimal transport
with the squared Euclidean cost, used to check the iteration and the exact
solvers against something other than themselves.

* 1D: for a convex cost on the line the monotone (north-west-corner on sorted
  supports, i.e. quantile) coupling is optimal.
* Product measures: if mu1 = p (x) q and mu2 = p' (x) q' on a grid, the cost
  (x_i - x_k)^2 + (y_j - y_l)^2 is separable and the product of the two optimal
  1D couplings is optimal, so W2^2 = W2^2(p, p') + W2^2(q, q').
* Integer translation: if mu2 is mu1 shifted by (s, t) then the translation
  map is the gradient of a convex function, hence optimal: W2^2 = s^2 + t^2.
"""
import numpy as np


def ot_1d(p, q, xs=None):
    """Quantile (monotone) coupling cost between histograms p, q on sorted points xs."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    xs = np.arange(p.size, dtype=np.float64) if xs is None else np.asarray(xs, dtype=np.float64)
    i = l = 0
    a, b = p[0], q[0]
    cost = 0.0
    while True:
        mv = min(a, b)
        cost += mv * (xs[i] - xs[l]) ** 2
        a -= mv
        b -= mv
        if a <= 0.0:
            i += 1
            if i == p.size:
                break
            a = p[i]
        if b <= 0.0:
            l += 1
            if l == q.size:
                break
            b = q[l]
    return cost


def product_measure_value(p, q, p2, q2, xs=None, ys=None):
    """W2^2 between p (x) q and p2 (x) q2 (rows x columns)."""
    return ot_1d(p, p2, xs) + ot_1d(q, q2, ys)


def translation_value(s, t):
    """W2^2 of an integer translation by (s, t)."""
    return float(s * s + t * t)


def brute_force_uniform(src_bins, dst_bins):
    """Exact W2^2 between two uniform measures on k bins each (k small):
    by Birkhoff's theorem an optimal plan is a permutation, so enumerate them."""
    import itertools
    src = np.asarray(src_bins, dtype=np.float64)
    dst = np.asarray(dst_bins, dtype=np.float64)
    k = len(src)
    C = ((src[:, None, :] - dst[None, :, :]) ** 2).sum(-1)
    best = np.inf
    for perm in itertools.permutations(range(k)):
        best = min(best, C[np.arange(k), perm].sum())
    return best / k
