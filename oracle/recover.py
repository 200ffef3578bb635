"""Algorithm 1 of arXiv 2408.00598: transport plan from the reduced-model flows.

Test infrastructure only (see ``oracle/__init__``).

Algorithm 1 loops over every intermediate node (k, j) and, for i = 1..m and
l = 1..n in that order, moves pi_{i,j;k,l} = min(f1_{i,k,j}, f2_{k,j,l}) and
subtracts it from both flows.  Prop. 1 shows the result is an optimal plan
when (f1, f2) is optimal.

Reading for an approximate solution (the paper assumes an exact optimum): the
loops run on the clipped flows max(f, 0); whatever a node cannot pass on
(conservation mismatch) stays unassigned and shows up as a marginal error;
zero entries are not emitted.
"""
import numpy as np

from .reduced_model import split_x


def recover_plan(f1, f2):
    """Literal Algorithm 1.  f1[i,k,j], f2[k,j,l] (0-based) -> list of
    (i, j, k, l, pi) with pi > 0, ordered by (k, j) then i then l."""
    f1 = np.array(f1, dtype=np.float64, copy=True)
    f2 = np.array(f2, dtype=np.float64, copy=True)
    m, _, n = f1.shape
    out = []
    for k in range(m):
        for j in range(n):
            for i in range(m):
                for l in range(n):
                    p = min(f1[i, k, j], f2[k, j, l])
                    f1[i, k, j] -= p
                    f2[k, j, l] -= p
                    if p > 0.0:
                        out.append((i, j, k, l, p))
    return out


def recover_cell(a, b):
    """Algorithm 1's two inner loops for one node (k, j): a = f1[:, k, j],
    b = f2[k, j, :] -> list of (i, l, pi) with pi > 0."""
    a = np.array(a, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    out = []
    for i in range(a.size):
        for l in range(b.size):
            p = min(a[i], b[l])
            a[i] -= p
            b[l] -= p
            if p > 0.0:
                out.append((i, l, p))
    return out


def recover_from_x(x, m, n):
    """Algorithm 1 on the clipped flows of a (possibly approximate) x = [f1; f2]."""
    f1, f2 = split_x(x, m, n)
    return recover_plan(np.maximum(f1, 0.0), np.maximum(f2, 0.0))


def plan_marginals(entries, m, n):
    """Row and column marginals of a plan given as (i, j, k, l, pi) entries."""
    r = np.zeros((m, n))
    s = np.zeros((m, n))
    for i, j, k, l, p in entries:
        r[i, j] += p
        s[k, l] += p
    return r, s


def plan_cost(entries, xs=None, ys=None):
    """sum pi_{ij;kl} ((x_i - x_k)^2 + (y_j - y_l)^2), eq. (1)-(2)."""
    tot = 0.0
    for i, j, k, l, p in entries:
        dx = (i - k) if xs is None else (xs[i] - xs[k])
        dy = (j - l) if ys is None else (ys[j] - ys[l])
        tot += p * (dx * dx + dy * dy)
    return tot
