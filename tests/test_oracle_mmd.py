"""Pins of the MMD oracle (paper Sec. 5, the MMD equation) to facts outside
itself: a hand-computed case, identical sets, point masses, a library l1
distance, and, for scalar embeddings, Cramer's identity (the statistic
equals 2 x the integral of the squared difference of the two empirical
distribution functions), which holds for the distance-based MMD and fails
for a dropped factor 2, a missing within-set term or a normalisation by
n (n - 1)."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import mmd as om


def test_hand_computed_case():
    """X = {0, 1}, Y = {2, 3}: sum d(x, y) = 2 + 3 + 1 + 2 = 8, sum d(x, x')
    = 2, sum d(y, y') = 2, so MMD = (2 * 8 - 2 - 2) / 4 = 3."""
    x = np.array([[0.0], [1.0]])
    y = np.array([[2.0], [3.0]])
    assert om.mmd(x, y) == 3.0
    d = om.l1_distances(np.vstack([x, y]))
    assert om.mmd_from_distances(d, [0, 1], [2, 3]) == 3.0


def test_identical_sets_and_point_masses():
    rng = np.random.default_rng(1)
    e = rng.standard_normal((6, 5))
    assert om.mmd(e, e) == 0.0
    a, b = rng.standard_normal(7), rng.standard_normal(7)
    # n copies of a against n copies of b: 2 d(a, b)
    got = om.mmd(np.tile(a, (4, 1)), np.tile(b, (4, 1)))
    assert got == pytest.approx(2.0 * np.abs(a - b).sum(), rel=1e-14)


def test_l1_distances_match_library_cityblock():
    rng = np.random.default_rng(2)
    e = rng.standard_normal((9, 33))
    assert np.allclose(om.l1_distances(e), cdist(e, e, metric="cityblock"), rtol=1e-14, atol=0)


def _cramer(x, y):
    """2 * integral over t of (F_x(t) - F_y(t))^2 for empirical CDFs."""
    pts = np.sort(np.concatenate([x, y]))
    total = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        fx = np.mean(x <= lo)
        fy = np.mean(y <= lo)
        total += (fx - fy) ** 2 * (hi - lo)
    return 2.0 * total


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_scalar_embeddings_obey_cramers_identity(seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(11)
    y = rng.standard_normal(11) * 1.5 + 0.4
    d = om.l1_distances(np.concatenate([x, y])[:, None])
    got = om.mmd_from_distances(d, np.arange(11), np.arange(11, 22))
    assert got == pytest.approx(_cramer(x, y), rel=1e-12)
    assert om.mmd(x[:, None], y[:, None]) == pytest.approx(got, rel=1e-12)
    # unequal sizes: the same identity
    d2 = om.l1_distances(np.concatenate([x[:7], y])[:, None])
    assert om.mmd_from_distances(d2, np.arange(7), np.arange(7, 18)) == pytest.approx(
        _cramer(x[:7], y), rel=1e-12)


def test_symmetric_nonnegative_and_trials():
    rng = np.random.default_rng(6)
    e = rng.standard_normal((20, 8))
    d = om.l1_distances(e)
    labels = np.full((3, 20), -1, dtype=np.int8)
    labels[0, :10], labels[0, 10:] = 0, 1
    labels[1, ::2], labels[1, 1::2] = 1, 0
    labels[2, :5], labels[2, 12:17] = 0, 1
    t = om.mmd_trials(d, labels)
    assert np.all(t >= 0)
    swapped = np.where(labels == 0, 1, np.where(labels == 1, 0, -1))
    assert np.allclose(om.mmd_trials(d, swapped), t, rtol=1e-14)
    assert t[0] == pytest.approx(om.mmd(e[:10], e[10:]), rel=1e-12)
