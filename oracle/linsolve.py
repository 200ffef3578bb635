"""Closed-form solution of AA^T y = R, Prop. 3 of arXiv 2408.00598 (Sec. III-B).

Test infrastructure only (see ``oracle/__init__``).

Block notation of eq. (equ:normal): y = (y1; y2; y3), R = (R1; R2; R3) with
y_i = (y_i^1; ...; y_i^n), each y_i^j in R^m, except y3^n and R3^n in R^{m-1}.
Block j of y1 / R1 holds the entries (k, j), k = 1..m (conservation rows);
block j of y2 / R2 holds (i, j) (mu1 rows); block l of y3 / R3 holds (k, l)
(mu2 rows).

Readings of garbled or ambiguous symbols in the printed proposition (each
checked against a dense solve of AA^T in the tests):

* "1_m^T y1^j" in eq. (y2) and "(1/n) 1_m^T R1^j", "1_m^T R2^j" in R~1^j, R~2^j
  are scalars; they are broadcast to m-vectors (times 1_m).
* In eq. (y3) the summation index j shadows the block index: the sum is
  s = sum_{j'=1}^{n} y1^{j'}, the same m-vector for every block; the last block
  takes Ibar_m s (its first m-1 entries).
* R~3 = (1/n)(sum_{j<n} R3^j + Ibar_m^T R3^n) + (1/n^2) 1_{M-1}^T R3, the last
  term a scalar broadcast to m entries.
* w = 1/m - (1 - 1/n)/(m + 1) > 0.
"""
import numpy as np


def split_blocks(R, m, n):
    """Split R (length 3mn - 1) into lists of blocks R1^j, R2^j, R3^j."""
    M = m * n
    R = np.asarray(R, dtype=np.float64)
    R1 = [R[m * j: m * (j + 1)] for j in range(n)]
    R2 = [R[M + m * j: M + m * (j + 1)] for j in range(n)]
    R3 = [R[2 * M + m * j: 2 * M + min(m * (j + 1), M - 1)] for j in range(n)]
    return R1, R2, R3


def solve_aat(R, m, n):
    """y with AA^T y = R by the formulas of Prop. 3; O(M3) flops (Cor. 1)."""
    R1, R2, R3 = split_blocks(R, m, n)
    one = np.ones(m)
    Ibar = np.eye(m)[: m - 1]                      # Ibar_m = [I_{m-1}, 0]

    # R~3 (item 1 of Prop. 3): one m-vector shared by all j.
    sumR3 = np.zeros(m)
    for j in range(n - 1):
        sumR3 += R3[j]
    sumR3 += Ibar.T @ R3[n - 1]
    total_R3 = sum(float(np.sum(R3[j])) for j in range(n))   # 1_{M-1}^T R3
    Rt3 = sumR3 / n + total_R3 / n ** 2

    # y1-hat^j = (R~1^j + R~2^j + R~3) / (m + n), item 1.
    y1_hat = []
    for j in range(n):
        Rt1 = R1[j] + (one @ R1[j]) / n * one
        Rt2 = -(1.0 / m + 1.0 / n) * (one @ R2[j]) * one
        y1_hat.append((Rt1 + Rt2 + Rt3) / (m + n))

    # W-hat, d and w (item 3).
    D = np.diag(np.concatenate([np.full(m - 1, 1.0 / m), [(1.0 - 1.0 / n) / (m + 1)]]))
    d = np.concatenate([np.full(m - 1, 1.0 / m), [(1.0 - 1.0 / n) / (m + 1)]])
    w = 1.0 / m - (1.0 - 1.0 / n) / (m + 1)
    W_hat = -D - np.outer(d, d) / w

    # y1-hat^a = (I_m + (1/n) 1 1^T) W-hat sum_j y1-hat^j (item 2).
    s_hat = np.zeros(m)
    for j in range(n):
        s_hat += y1_hat[j]
    y1_a = (np.eye(m) + np.outer(one, one) / n) @ (W_hat @ s_hat)

    # eq. (y1), (y2), (y3).
    y1 = [y1_hat[j] - y1_a for j in range(n)]
    y2 = [(R2[j] - (one @ y1[j]) * one) / m for j in range(n)]
    s = np.zeros(m)
    for j in range(n):
        s += y1[j]
    y3 = [(R3[j] + s) / n for j in range(n - 1)]
    y3.append((R3[n - 1] + Ibar @ s) / n)
    return np.concatenate(y1 + y2 + y3)
