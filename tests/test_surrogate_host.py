"""Host-side bookkeeping of the surrogate search (no GPU): the fixed input
standardisation, the candidate draws over the search box, the best-so-far curve and the
evaluation count at which a target is first met."""
import math

import numpy as np

from paper_2404_12454_gb300 import surrogate as S
from paper_2404_12454_gb300 import workloads as W


def test_standardisation_gives_zero_mean_unit_variance_over_the_box():
    """The fixed affine map is the standardisation of the search box's own distributions
    (OF ~ U[1, 3], WR ~ U[0.8, 3], log2 N uniform on 4..8): the corners land on +-sqrt(3)
    (the uniform inputs) and +-sqrt(2) (log2 N), and a large draw has mean 0 and standard
    deviation 1 per feature."""
    corners = [(n, of, wr) for n in (16, 256) for of in (1.0, 3.0) for wr in (0.8, 3.0)]
    z = S.standardize(corners)
    assert z.shape == (8, 3) and z.dtype == np.float32
    assert np.allclose(np.abs(z[:, :2]), math.sqrt(3.0), rtol=1e-3)
    assert np.allclose(np.abs(z[:, 2]), math.sqrt(2.0), rtol=1e-3)
    assert np.allclose(S.standardize([(64, 2.0, 1.9)])[0], 0.0, atol=1e-6)
    d = S.standardize(S.random_candidates(200000, np.random.default_rng(1)))
    assert np.allclose(d.mean(axis=0), 0.0, atol=0.01)
    assert np.allclose(d.std(axis=0), 1.0, atol=0.01)


def test_random_candidates_stay_in_the_box_and_are_seeded():
    a = S.random_candidates(5000, np.random.default_rng(3))
    b = S.random_candidates(5000, np.random.default_rng(3))
    assert a == b
    n = np.array([p[0] for p in a])
    of = np.array([p[1] for p in a])
    wr = np.array([p[2] for p in a])
    assert set(np.unique(n)) == set(W.SWEEP_N_ACROSS)
    assert of.min() >= 1.0 and of.max() < 3.0 and wr.min() >= 0.8 and wr.max() < 3.0
    # uniform: every fifth of each range is drawn about as often
    for v, lo, hi in ((of, 1.0, 3.0), (wr, 0.8, 3.0)):
        h, _ = np.histogram(v, bins=5, range=(lo, hi))
        assert h.min() > 0.8 * len(v) / 5


def test_best_so_far_curve_and_evaluations_to_target():
    scores = [5.0, 4.0, 6.0, 3.0, 3.5, 2.0, 9.0]
    steps = [2, 3, 2]
    curve = S._curve(np.asarray(scores), steps)
    assert curve == [(2, 4.0), (5, 3.0), (7, 2.0)]
    res = S.SearchResult([(16, 1.0, 1.0)] * 7, scores, curve)
    assert res.best == ((16, 1.0, 1.0), 2.0)
    assert res.evals_to_reach(4.0) == 2
    assert res.evals_to_reach(3.0) == 5
    assert res.evals_to_reach(2.5) == 7
    assert res.evals_to_reach(1.0) is None
    # a curve never rises, and its last point is the overall minimum
    rng = np.random.default_rng(0)
    s = rng.uniform(size=100)
    c = S._curve(s, [10] * 10)
    assert all(c[k + 1][1] <= c[k][1] for k in range(len(c) - 1))
    assert c[-1] == (100, float(s.min()))
    assert math.isclose(c[0][1], float(s[:10].min()))
