"""The seeded input generators (shared by tests, bench and oracle callers)."""
import numpy as np
import pytest

from paper_2408_00598_gb300 import synthetic as syn


@pytest.mark.parametrize("kind", syn.KINDS)
@pytest.mark.parametrize("S", [16, 33, 64])
def test_pairs_are_histograms_and_deterministic(kind, S):
    a1, b1 = syn.make_pair(kind, S, 5)
    a2, b2 = syn.make_pair(kind, S, 5)
    for a in (a1, b1):
        assert a.shape == (S, S) and a.dtype == np.float64
        assert a.min() >= 0.0
        assert abs(a.sum() - 1.0) < 1e-12
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(b1, b2)


def test_translation_is_a_shift():
    for seed in range(5):
        mu1, mu2, s, t = syn.make_translation(32, seed)
        shifted = np.zeros_like(mu1)
        m, n = mu1.shape
        for i in range(m):
            for j in range(n):
                if mu1[i, j] > 0:
                    shifted[i + s, j + t] = mu1[i, j]
        np.testing.assert_allclose(shifted, mu2, atol=1e-18)
        assert 1 <= s * s + t * t <= 2 * 16


def test_mixed_batch():
    batch = syn.mixed_batch([32, 48, 64], 20, 1)
    assert len(batch) == 20
    assert {b[1] for b in batch} <= {32, 48, 64}


@pytest.mark.parametrize("kind", syn.KINDS)
@pytest.mark.parametrize("m,n", [(8, 12), (20, 8), (24, 72)])
def test_rectangular_pairs(kind, m, n):
    a, b = syn.make_pair(kind, m, 3, n=n)
    for h in (a, b):
        assert h.shape == (m, n) and h.min() >= 0.0
        assert abs(h.sum() - 1.0) < 1e-12
