"""Pins of the oracle's plan consumer (barycentric projection, the colour-
transfer use of a plan, Sec. IV-B / App. G)."""
import numpy as np

from oracle import consumers, exact, hot, recover
from paper_2408_00598_gb300 import synthetic as syn


def test_barycentric_map_by_hand():
    # source 0 sends 0.25 to target 1 and 0.75 to target 2; source 1 all to 0;
    # source 2 ships nothing
    src, dst, mass = [0, 0, 1], [1, 2, 0], [0.25, 0.75, 0.5]
    y = np.array([[0.0, 0.0], [4.0, 8.0], [8.0, 0.0]])
    out, w = consumers.barycentric_map(src, dst, mass, y, 3)
    np.testing.assert_allclose(out[0], [0.25 * 4 + 0.75 * 8, 0.25 * 8])
    np.testing.assert_allclose(out[1], [0.0, 0.0])
    np.testing.assert_allclose(w, [1.0, 0.5, 0.0])
    np.testing.assert_array_equal(out[2], [0.0, 0.0])


def test_identity_plan_maps_every_bin_to_itself():
    rng = np.random.default_rng(3)
    n = 7
    mass = rng.uniform(0.1, 1.0, n)
    y = rng.standard_normal((n, 3))
    out, w = consumers.barycentric_map(np.arange(n), np.arange(n), mass, y, n)
    np.testing.assert_allclose(out, y, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, mass)


def test_translation_plan_maps_bins_by_the_shift():
    """The optimal plan between a measure and its integer translate by (s, t)
    moves every bin by (s, t) (the closed form s^2 + t^2 of the value is
    attained only by that plan on these supports), so the barycentric image of
    every source bin with mass is its own coordinate plus (s, t)."""
    S = 8
    mu1, mu2, s, t = syn.make_translation(S, 4)
    r = hot.hot_solve(mu1, mu2, tol=1e-11, max_iter=400000)
    plan = recover.recover_from_x(r.x, S, S)
    src = [i * S + j for i, j, k, l, p in plan]
    dst = [k * S + l for i, j, k, l, p in plan]
    mass = [p for *_, p in plan]
    xy = consumers.grid_coordinates(S, S)
    out, w = consumers.barycentric_map(src, dst, mass, xy, S * S)
    has = mu1.ravel() > 1e-9
    np.testing.assert_allclose(w[has], mu1.ravel()[has], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(out[has], xy[has] + np.array([s, t]), rtol=0, atol=1e-4)


def test_grid_coordinates_are_row_major():
    xy = consumers.grid_coordinates(2, 3)
    np.testing.assert_array_equal(xy, [[0, 0], [0, 1], [0, 2], [1, 0], [1, 1], [1, 2]])
