"""The reduced OT model and its standard LP form (Sec. II-A of arXiv 2408.00598).

Test infrastructure only (see ``oracle/__init__``).

Indexing.  The histograms live on an m x n grid; bin (i, j) has row i and
column j (0-based here, 1-based in the paper).  Eq. (6) builds A from Kronecker
products, which fixes the vec order of every vector:

* a histogram mu is vec'd column-major, row index innermost: entry (i, j) sits
  at i + m*j;
* f1_{i,k,j} (eq. 3: flow from bin (i,j) to bin (k,j) along column j) sits at
  i + m*k + m*m*j  ([j][k][i], i innermost), because A1 = I_M kron 1_m^T sums
  m consecutive entries and A3 = I_n kron (1_m^T kron I_m) sums entries m apart;
* f2_{k,j,l} (flow from bin (k,j) to bin (k,l) along row k) sits at
  k + m*j + m*n*l  ([l][j][k], k innermost), because A2 = -1_n^T kron I_M sums
  entries M apart and A4hat = I_n kron (1_n^T kron I_m) groups them by l.

The constraint rows are, in order: (k,j) conservation rows (A1, A2; index
k + m*j), mu1 rows (A3; index i + m*j), mu2 rows (A4; index k + m*l, the last
one, (m-1, n-1), dropped as in eq. (7)-(8)).
"""
import numpy as np
import scipy.sparse as sp


def vec(mu):
    """Column-major vec of an m x n histogram: entry (i, j) -> i + m*j (eq. 6)."""
    return np.asarray(mu, dtype=np.float64).T.reshape(-1)


def unvec(v, m, n):
    """Inverse of ``vec``."""
    return np.asarray(v).reshape(n, m).T


def f1_index(i, k, j, m, n):
    """Position of f1_{i,k,j} in x (eq. 4, ordering forced by eq. 6)."""
    return i + m * k + m * m * j


def f2_index(k, j, l, m, n):
    """Position of f2_{k,j,l} in x: offset m^2 n plus k + m*j + m*n*l (eq. 4, 6)."""
    return m * m * n + k + m * j + m * n * l


def _ones_row(k):
    return sp.csr_matrix(np.ones((1, k)))


def build_A_hat(m, n):
    """A-hat of eq. (4) with the blocks of eq. (6); shape (3M) x (m^2 n + m n^2)."""
    M = m * n
    I = lambda k: sp.identity(k, format="csr")
    A1 = sp.kron(I(M), _ones_row(m))                    # I_M kron 1_m^T
    A2 = -sp.kron(_ones_row(n), I(M))                   # -1_n^T kron I_M
    A3 = sp.kron(I(n), sp.kron(_ones_row(m), I(m)))     # I_n kron (1_m^T kron I_m)
    A4h = sp.kron(I(n), sp.kron(_ones_row(n), I(m)))    # I_n kron (1_n^T kron I_m)
    Z13 = sp.csr_matrix((M, m * n * n))
    Z31 = sp.csr_matrix((M, m * m * n))
    return sp.vstack([sp.hstack([A1, A2]),
                      sp.hstack([A3, Z13]),
                      sp.hstack([Z31, A4h])]).tocsr()


def build_A(m, n):
    """Full-row-rank A of eq. (7)-(8): A-hat with its last row (the (m, n) entry
    of the mu2 block) removed, i.e. A4 = diag(1_n^T kron I_m, ..., 1_n^T kron Ibar_m)."""
    Ah = build_A_hat(m, n)
    return Ah[: 3 * m * n - 1].tocsr()


def build_b(mu1, mu2):
    """b = [0_M; mu1; Ibar_M mu2] of eq. (7) (the last mu2 entry dropped)."""
    m, n = np.shape(mu1)
    M = m * n
    return np.concatenate([np.zeros(M), vec(mu1), vec(mu2)[: M - 1]])


def build_b_hat(mu1, mu2):
    """b-hat = [0_M; mu1; mu2] of eq. (4)."""
    m, n = np.shape(mu1)
    return np.concatenate([np.zeros(m * n), vec(mu1), vec(mu2)])


def grid_coords(m, n, xs=None, ys=None):
    """Row coordinates x_0..x_{m-1} and column coordinates y_0..y_{n-1}.

    Eq. (2) uses the bin indices themselves; non-uniform bins (Sec. IV-B, App. E)
    replace them by arbitrary increasing coordinates."""
    xs = np.arange(m, dtype=np.float64) if xs is None else np.asarray(xs, dtype=np.float64)
    ys = np.arange(n, dtype=np.float64) if ys is None else np.asarray(ys, dtype=np.float64)
    return xs, ys


def build_c(m, n, xs=None, ys=None):
    """c = [c1; c2] of eq. (4): c1_{i,k,j} = (k - i)^2, c2_{k,j,l} = (j - l)^2
    (with coordinates: (x_k - x_i)^2 and (y_j - y_l)^2)."""
    xs, ys = grid_coords(m, n, xs, ys)
    c = np.empty(m * m * n + m * n * n)
    for j in range(n):
        for k in range(m):
            for i in range(m):
                c[f1_index(i, k, j, m, n)] = (xs[k] - xs[i]) ** 2
    for l in range(n):
        for j in range(n):
            for k in range(m):
                c[f2_index(k, j, l, m, n)] = (ys[j] - ys[l]) ** 2
    return c


def full_cost_matrix(m, n, xs=None, ys=None):
    """Cost c_{ij;kl} of eq. (2) with p = 2, as an M x M matrix indexed by the
    vec positions i + m*j (source bin) and k + m*l (target bin)."""
    xs, ys = grid_coords(m, n, xs, ys)
    M = m * n
    C = np.empty((M, M))
    for j in range(n):
        for i in range(m):
            for l in range(n):
                for k in range(m):
                    C[i + m * j, k + m * l] = (xs[i] - xs[k]) ** 2 + (ys[j] - ys[l]) ** 2
    return C


def aat_blocks(m, n):
    """Dense E1..E5 of eq. (Mat:OT_AAT), written from their printed definitions."""
    M = m * n
    E1 = (m + n) * np.eye(M)
    E2 = np.kron(np.eye(n), np.ones((m, m)))
    Ibar = np.eye(m)[: m - 1]
    blocks = [np.eye(m)] * (n - 1) + [Ibar.T]
    E3 = -np.kron(np.ones((n, 1)), np.hstack(blocks))
    E4 = m * np.eye(M)
    E5 = n * np.eye(M - 1)
    return E1, E2, E3, E4, E5


def aat_from_blocks(m, n):
    """Assemble AA^T of eq. (Mat:OT_AAT) from the E blocks."""
    E1, E2, E3, E4, E5 = aat_blocks(m, n)
    M = m * n
    Z24 = np.zeros((M, M - 1))
    return np.block([[E1, E2, E3], [E2.T, E4, Z24], [E3.T, Z24.T, E5]])


def split_x(x, m, n):
    """Return f1[i,k,j] and f2[k,j,l] (0-based) from x = [f1; f2]."""
    x = np.asarray(x)
    f1 = x[: m * m * n].reshape(n, m, m).transpose(2, 1, 0)     # [j][k][i] -> [i][k][j]
    f2 = x[m * m * n:].reshape(n, n, m).transpose(2, 1, 0)      # [l][j][k] -> [k][j][l]
    return f1, f2
