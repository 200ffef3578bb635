"""Seeded synthetic histogram pairs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the CPU oracle's callers;
it holds no part of the solver's arithmetic, only input generation.

The paper evaluates on DOTmark (Classic images and Shapes, resized to
64^2 ... 512^2, Sec. IV-A), which is not available here; these classes stand
in for it.  Every generator draws from ``numpy.random.default_rng(seed)``
(PCG64) and returns two m x n float64 arrays, each non-negative and
normalised to total mass 1 in float64.  Rows are the first index i, columns
the second index j, row-major in memory.

Classes (``KINDS``):

* ``white``     i.i.d. Uniform(0.1, 1) entries.
* ``gauss``     1-8 isotropic Gaussian bumps, centres uniform over the grid,
                std Uniform(2, 12) px, weights Uniform(0.5, 1), plus a 1e-6
                floor (smooth images, like DOTmark Classic).
* ``cauchy``    (1 + r^2/gamma^2)^(-alpha), random centre, gamma in
                Uniform(1, max(1, S/8)), alpha in Uniform(0.75, 1.5)
                (heavy-tailed density).
* ``shapes``    1-6 axis-aligned rectangles or ellipses with levels
                Uniform(0.2, 1) on a zero background (like DOTmark Shapes;
                exact zeros allowed).
* ``translate`` mu1 from one of the classes above restricted to the box
                [0, m-1-|s|] x [0, n-1-|t|] (placed so the shift stays on the
                grid), mu2 = mu1 shifted by integers (s, t) with |s|, |t| <=
                max(1, S/8); the exact answer is s^2 + t^2.
"""
import numpy as np

KINDS = ("white", "gauss", "cauchy", "shapes", "translate")


def _normalise(a):
    a = np.asarray(a, dtype=np.float64)
    s = a.sum()
    if s <= 0.0:
        a = np.zeros_like(a)
        a[a.shape[0] // 2, a.shape[1] // 2] = 1.0
        return a
    return a / s


def _white(rng, m, n):
    return rng.uniform(0.1, 1.0, (m, n))


def _gauss(rng, m, n):
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    out = np.full((m, n), 1e-6)
    for _ in range(int(rng.integers(1, 9))):
        ci, cj = rng.uniform(0, m), rng.uniform(0, n)
        sd = rng.uniform(2.0, 12.0)
        wgt = rng.uniform(0.5, 1.0)
        out += wgt * np.exp(-((ii - ci) ** 2 + (jj - cj) ** 2) / (2.0 * sd * sd))
    return out


def _cauchy(rng, m, n):
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    S = max(m, n)
    ci, cj = rng.uniform(0, m), rng.uniform(0, n)
    gamma = rng.uniform(1.0, max(1.0, S / 8.0) + 1e-9)
    alpha = rng.uniform(0.75, 1.5)
    r2 = (ii - ci) ** 2 + (jj - cj) ** 2
    return (1.0 + r2 / gamma ** 2) ** (-alpha)


def _shapes(rng, m, n):
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    out = np.zeros((m, n))
    for _ in range(int(rng.integers(1, 7))):
        ci, cj = rng.uniform(0, m), rng.uniform(0, n)
        ri = rng.uniform(max(1.0, m / 16), max(1.5, m / 3))
        rj = rng.uniform(max(1.0, n / 16), max(1.5, n / 3))
        lev = rng.uniform(0.2, 1.0)
        if rng.random() < 0.5:
            mask = (np.abs(ii - ci) <= ri) & (np.abs(jj - cj) <= rj)
        else:
            mask = ((ii - ci) / ri) ** 2 + ((jj - cj) / rj) ** 2 <= 1.0
        out[mask] = np.maximum(out[mask], lev)
    return out


_BASE = {"white": _white, "gauss": _gauss, "cauchy": _cauchy, "shapes": _shapes}


def translate_pair(rng, m, n, base_kind=None):
    """(mu1, mu2, s, t): mu2 is mu1 moved by (s, t) rows/columns."""
    S = max(m, n)
    smax = max(1, S // 8)
    s = int(rng.integers(-smax, smax + 1))
    t = int(rng.integers(-smax, smax + 1))
    if s == 0 and t == 0:
        s = 1
    kind = base_kind or ("white", "gauss", "cauchy", "shapes")[int(rng.integers(0, 4))]
    mh, nh = m - abs(s), n - abs(t)
    sub = _BASE[kind](rng, mh, nh)
    mu1 = np.zeros((m, n))
    mu2 = np.zeros((m, n))
    i0 = max(0, -s)
    j0 = max(0, -t)
    mu1[i0:i0 + mh, j0:j0 + nh] = sub
    mu2[i0 + s:i0 + s + mh, j0 + t:j0 + t + nh] = sub
    return _normalise(mu1), _normalise(mu2), s, t


def make_pair(kind, m, seed, n=None):
    """Two m x n histograms of class ``kind`` from ``seed`` (see module docstring)."""
    n = m if n is None else n
    rng = np.random.default_rng(int(seed))
    if kind == "translate":
        mu1, mu2, _, _ = translate_pair(rng, m, n)
        return mu1, mu2
    if kind not in _BASE:
        raise ValueError("unknown kind %r" % (kind,))
    return _normalise(_BASE[kind](rng, m, n)), _normalise(_BASE[kind](rng, m, n))


def make_translation(m, seed, n=None, base_kind=None):
    """(mu1, mu2, s, t) of the ``translate`` class."""
    n = m if n is None else n
    return translate_pair(np.random.default_rng(int(seed)), m, n, base_kind)


def mixed_batch(sizes, count, seed):
    """``count`` pairs with S drawn uniformly from ``sizes`` and classes drawn
    uniformly from KINDS: list of (kind, S, pair_seed, mu1, mu2)."""
    rng = np.random.default_rng(int(seed))
    out = []
    for q in range(count):
        S = int(sizes[int(rng.integers(0, len(sizes)))])
        kind = KINDS[int(rng.integers(0, len(KINDS)))]
        pseed = int(seed) * 100003 + q
        mu1, mu2 = make_pair(kind, S, pseed)
        out.append((kind, S, pseed, mu1, mu2))
    return out
