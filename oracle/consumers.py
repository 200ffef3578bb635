"""Consumers of a recovered transport plan (Sec. IV-B, App. G: colour transfer).

Test infrastructure only (see ``oracle/__init__``).

A plan from Algorithm 1 is a list of entries (s, t, pi): mass pi moved from
source bin s to target bin t.  Colour transfer (and any dense use of an OT
plan) applies its barycentric projection: each source bin s is sent to the
pi-weighted mean of the target values y_t it ships mass to,

    T(s) = sum_t pi(s, t) y_t / sum_t pi(s, t),

with y_t a D-vector per target bin (a colour, or the bin's coordinates).
Source bins that ship no mass have no image; they are reported with weight 0
and value 0.
"""
import numpy as np


def barycentric_map(src, dst, mass, y, nsrc):
    """T(s) for s < nsrc and the row weights sum_t pi(s, t) (plain definition,
    one pass over the entries in order)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    mass = np.asarray(mass, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if y.ndim == 1:
        y = y[:, None]
    num = np.zeros((nsrc, y.shape[1]))
    w = np.zeros(nsrc)
    for s, t, p in zip(src, dst, mass):
        num[s] += p * y[t]
        w[s] += p
    out = np.zeros_like(num)
    nz = w > 0
    out[nz] = num[nz] / w[nz, None]
    return out, w


def grid_coordinates(m, n):
    """(i, j) coordinates of the bins of an m x n grid in row-major bin order."""
    i, j = np.meshgrid(np.arange(m, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    return np.stack([i.ravel(), j.ravel()], axis=1)
