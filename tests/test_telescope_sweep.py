"""The parameter search on the App. B telescope: batched sweeps whose instances are traced
by real rays through the two conic mirrors (gbd_sweep_plan_create_mirrors), against the
oracle's own mirror trace, field and Airy score; then the surrogate against random search
on that landscape.

Scores are compared relatively, to 1e-3 of the oracle's score, the bound derived in
tests/test_sweep.py (measured on the 1024-instance sweep's six instances where the row
pairs and the row triples differ most, all 256 across: pairs within 9e-5, triples with
per-column row factors within 2.2e-4).  The image plane
is the real system's least-RMS focus (workloads.HST_REFOCUS), where the score measures the
decomposition: on this landscape the 1 % window around the grid optimum (256 across,
OF 1.0) is OF below ~1.15 at 256 across, about 1.5 % of the search box.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCORE_RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_12454_gb300 import build
    build.build()
    import torch
    torch.cuda.init()


def oracle_scores(sw, idx):
    """Oracle Airy scores of MirrorSweep instances, the field evaluated on the square of
    pixels that holds the scored disc."""
    det = sw.detector
    lam, F = sw.system.wavelength, sw.f_number
    r3 = 10.173468135062722 * lam * F / math.pi
    h = min(int(math.ceil(r3 / det.pitch_x)) + 1, det.nx // 2 - 1)
    cols = rows = np.arange(det.nx // 2 - h, det.nx // 2 + h + 1)
    out = []
    for k in idx:
        b = oracle.trace_mirrors(sw.system, sw.pupil(k))
        E = np.zeros((det.ny, det.nx), dtype=np.complex128)
        E[np.ix_(rows, cols)] = oracle.field(b, sw.system, det, cols=cols, rows=rows)
        out.append(oracle.airy_score(E, det, lam, F))
    return np.array(out)


def assert_scores(got, want):
    rel = np.abs(np.asarray(got) - want) / want
    assert np.all(np.isfinite(got)) and np.max(rel) <= SCORE_RTOL, (np.max(rel), got, want)


def test_full_telescope_sweep_seeded_subset_matches_oracle():
    """The 1024 seeded instances traced through the telescope in one batched trace and one
    persistent field + score launch; 14 re-scored by the oracle (3 of each beamlet count up
    to 128, the two 256-across instances with the smallest overlap factors)."""
    sw = W.telescope_sweep()
    plan = gbd.sweep_plan(sw)
    got = plan.run().cpu().numpy()
    gbd.gbd_sync()
    assert np.all(np.isfinite(got)) and plan.n == 1024
    n = np.asarray(sw.n_across)
    rng = np.random.default_rng(240412455)
    idx = []
    for N in (16, 32, 64, 128):
        idx += list(rng.choice(np.flatnonzero(n == N), size=3, replace=False))
    c256 = np.flatnonzero(n == 256)
    idx += list(c256[np.argsort(np.asarray(sw.overlap_factor)[c256])[:2]])
    assert_scores(got[idx], oracle_scores(sw, idx))


@pytest.mark.parametrize("shape", [None, (3, 8, 1), (2, 4, gbd.GBD_SCHEME_ROW_PAIR), (2, 4, 0)])
def test_telescope_sweep_shapes_match_oracle(shape):
    """Every sweep shape on telescope instances up to 256 across (the real-ray fields have a
    uv term: the mirror default runs the 2 x 8 row pairs, the row triples their
    instantiation with per-column row factors, folding their FP32 sums into the compensated
    pair after every tile)."""
    params = [(16, 1.3, 0.9), (32, 2.4, 2.5), (64, 1.1, 1.0), (48, 1.7, 3.0), (256, 1.0, 1.0)]
    sw = W.telescope_sweep_from_params(params)
    got = gbd.sweep_plan(sw, shape=shape).run().cpu().numpy()
    gbd.gbd_sync()
    assert_scores(got, oracle_scores(sw, range(len(params))))


def test_telescope_grid_optimum_neighbourhood_is_ranked_like_the_oracle():
    """At 256 across the scores rise with the overlap factor (1.0, 1.1, 1.2 differ by
    0.6 %); the sweep orders them as the oracle does, and the waist ratio changes the score
    by less than 1e-4 relative (the parabasal steps are small against the mirrors'
    curvature, so the differential trace barely depends on them)."""
    params = [(256, of, 1.0) for of in (1.0, 1.1, 1.2)] + [(256, 1.0, 3.0)]
    sw = W.telescope_sweep_from_params(params)
    got = gbd.sweep_plan(sw).run().cpu().numpy()
    gbd.gbd_sync()
    want = oracle_scores(sw, [0, 1, 2])
    assert_scores(got[:3], want)
    assert np.all(np.diff(want) > 0) and np.array_equal(np.argsort(got[:3]), np.argsort(want))
    assert abs(got[3] - got[0]) <= 1e-4 * got[0]


def test_surrogate_needs_fewer_evaluations_than_random_search_on_the_telescope():
    """Evaluations to come within 1 % and within 0.1 % of the telescope grid's optimum,
    from the same seeded 32 random draws, then 32 per round (surrogate proposals / further
    random draws), capped at the grid's 1,260 (counted as 1,260); mean over 8 seeds.  The
    grid's optimum is (256 across, OF 1.0): the score rises with OF at every beamlet count."""
    from paper_2404_12454_gb300 import surrogate as S
    optics = W.telescope_sweep_from_params
    grid = S.grid_search(optics=optics)
    (N, of, wr), best = grid.best
    assert N == 256 and of == 1.0
    for tol, factor in ((1.01, 1.0), (1.001, 0.5)):
        res = S.compare_with_random(tol * best, seeds=range(8), optics=optics)
        sur = [v if v is not None else 1260 for v in res["surrogate"]]
        rnd = [v if v is not None else 1260 for v in res["random"]]
        assert np.mean(sur) < factor * np.mean(rnd), (tol, sur, rnd)
