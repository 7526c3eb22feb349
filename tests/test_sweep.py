"""Batched parameter sweep (persistent kernel with fused Airy score) against the oracle.

The oracle scores an instance by tracing it, summing its field on every pixel in FP64 and
applying the score's definition directly.  The sweep computes the mixed-precision field and
the score from moments.  A field error of relative L2 eps moves the score by at most about
2 eps (the score is an RMS over fewer pixels than the field's norm), so the bound here is
2 x the mixed-path tolerance, 4e-5.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCORE_TOL = 4e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_12454_gb300 import build
    build.build()
    import torch
    torch.cuda.init()


def oracle_scores(sw, idx):
    out = []
    for k in idx:
        pupil = sw.pupil(k)
        b = oracle.trace(sw.system, pupil)
        E = oracle.field(b, sw.system, sw.detector)
        out.append(oracle.airy_score(E, sw.detector, sw.system.wavelength,
                                     sw.system.focal_length / sw.diameter))
    return np.array(out)


def small_sweep():
    rng = np.random.default_rng(7)
    n = [16, 32, 64, 16, 32, 128, 64, 32, 16, 64]
    of = rng.uniform(1.0, 3.0, size=len(n))
    wr = rng.uniform(0.8, 3.0, size=len(n))
    return W.sweep_from_params(list(zip(n, of, wr)))


def test_small_sweep_scores_match_oracle():
    sw = small_sweep()
    plan = gbd.sweep_plan(sw)
    got = plan.run().cpu().numpy()
    gbd.gbd_sync()
    want = oracle_scores(sw, range(sw.n_instances))
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - want)) <= SCORE_TOL, (got, want)
    # the scores are distinct numbers, not a constant
    assert np.ptp(want) > 1e-3


def test_sweep_deterministic_graph_and_shapes():
    import torch
    sw = small_sweep()
    plan = gbd.sweep_plan(sw)
    a = plan.run().clone()
    b = plan.run().clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = plan.run(stream=s, graph=True).clone()
        d = plan.run(stream=s, graph=True).clone()
    s.synchronize()
    gbd.gbd_sync()
    assert torch.equal(a, b) and torch.equal(a, c) and torch.equal(c, d)
    for shape in ((1, 4), (2, 2), (2, 4), (4, 2), (2, 4, gbd.GBD_SCHEME_ROW_PAIR),
                  (2, 8, gbd.GBD_SCHEME_ROW_PAIR), (3, 8, gbd.GBD_SCHEME_ROW_PAIR)):
        p2 = gbd.sweep_plan(sw, shape=shape)
        e = p2.run().clone()
        gbd.gbd_sync()
        assert torch.max(torch.abs(e - a)).item() < 1e-6, shape


def test_full_sweep_seeded_subset_matches_oracle():
    """The 1024-instance sweep in one persistent launch (default shape: 3 x 8 row triples);
    16 seeded instances re-scored by the oracle (chosen across every beamlet count, at
    most one of 256 across)."""
    sw = W.sweep()
    plan = gbd.sweep_plan(sw)
    assert plan.n == 1024 and plan.items == 1024 * 11  # default blocks: 256 x 24 pixels
    got = plan.run().cpu().numpy()
    gbd.gbd_sync()
    assert np.all(np.isfinite(got))
    n = np.asarray(sw.n_across)
    rng = np.random.default_rng(240412455)
    idx = []
    for N, count in ((16, 4), (32, 4), (64, 4), (128, 3), (256, 1)):
        cand = np.flatnonzero(n == N)
        idx += list(rng.choice(cand, size=count, replace=False))
    want = oracle_scores(sw, idx)
    assert np.max(np.abs(got[idx] - want)) <= SCORE_TOL, (got[idx], want)


def test_sweep_autotune_picks_a_supported_shape():
    import torch
    sw = W.sweep_subset(W.sweep(), list(range(24)))
    probe = gbd.sweep_plan(sw, shape=(2, 8, gbd.GBD_SCHEME_ROW_PAIR))
    ws = torch.empty(probe.bytes * 2, dtype=torch.uint8, device="cuda")
    scores = torch.empty(sw.n_instances, dtype=torch.float64, device="cuda")
    r, c, ms, scheme = gbd.gbd_sweep_autotune(sw.system, sw.diameter, sw.n_across,
                                              sw.overlap_factor, sw.waist_ratio, sw.detector,
                                              ws, scores)
    assert (r, c, scheme) in ((1, 4, 0), (2, 2, 0), (2, 4, 0), (4, 2, 0), (2, 4, 1),
                              (2, 8, 1), (3, 8, 1)) and ms > 0


def test_sweep_rejects_bad_instances():
    sw = small_sweep()
    with pytest.raises(gbd.GbdError):
        gbd.SweepPlan(sw.system, sw.diameter, [16, 0], [1.5, 1.5], [1.0, 1.0], sw.detector)
    with pytest.raises(gbd.GbdError):
        gbd.SweepPlan(sw.system, sw.diameter, [16], [-1.0], [1.0], sw.detector)
    with pytest.raises(gbd.GbdError):
        gbd.SweepPlan(W.System(1e-6, math.inf, 0.02), sw.diameter, [16], [1.5], [1.0],
                      sw.detector)


def test_sweep_timeout_reported_then_recovers():
    sw = small_sweep()
    plan = gbd.sweep_plan(sw)
    ref = plan.run().clone()
    gbd.gbd_sync()
    try:
        gbd.gbd_set_wait_limit(1)
        plan.run()
        with pytest.raises(gbd.GbdError) as ei:
            gbd.gbd_sync()
        assert ei.value.status == gbd.GBD_ETIMEOUT
    finally:
        gbd.gbd_set_wait_limit(0)
    again = plan.run().clone()
    gbd.gbd_sync()
    assert bool((again == ref).all())


def test_zone_scores_match_oracle():
    """Annular zones of Sec. 6 (0-5, 5-10, 10-15 lambda/D) fused into the sweep epilogue,
    on a 512x512 detector over +-15.2 lambda F#."""
    full = W.zone_sweep()
    sw = W.sweep_subset(full, [0, 5, 10, 13, 18])
    plan = gbd.sweep_plan(sw, zones=W.ANNULAR_ZONES)
    got = plan.run().cpu().numpy()
    gbd.gbd_sync()
    assert got.shape == (5, 4)
    lam, F = sw.system.wavelength, sw.system.focal_length / sw.diameter
    for k in range(sw.n_instances):
        b = oracle.trace(sw.system, sw.pupil(k))
        E = oracle.field(b, sw.system, sw.detector)
        want = [oracle.airy_score(E, sw.detector, lam, F)]
        want += [oracle.zone_score(E, sw.detector, lam, F, lo, hi) for lo, hi in W.ANNULAR_ZONES]
        assert np.max(np.abs(got[k] - np.asarray(want))) <= SCORE_TOL, (k, got[k], want)
    # the plain score column equals a plan without zones
    plain = gbd.sweep_plan(sw).run().cpu().numpy()
    assert np.array_equal(plain, got[:, 0])


@pytest.mark.parametrize("shape", [None, (2, 8, 1), (3, 8, 1)])
def test_sweep_row_recurrences_fall_back_on_steep_beamlets(shape):
    """Beamlets 2.5 pixels wide on a coarse 96-pixel detector: the projection flags them as
    too steep for the row recurrences and the row-pair and row-triple plans evaluate them
    directly; scores match the oracle's."""
    system, D, _ = W.sweep_optics()
    det = W.Detector(96, 96, 1e-5, 1e-5)
    sw = W.Sweep(system, D, det, (4, 6), (1.0, 1.2), (1.0, 1.5))
    got = gbd.sweep_plan(sw, shape=shape).run().cpu().numpy()
    gbd.gbd_sync()
    want = oracle_scores(sw, range(sw.n_instances))
    assert np.max(np.abs(got - want)) <= SCORE_TOL, (got, want)


@pytest.mark.parametrize("shape", [None, (2, 8, 1)])
def test_sweep_general_row_pair_instantiation(shape):
    """A coarse detector (4 um pixels, +-25 lambda F#) where the beamlets are narrower than
    a thread's column span: the projection flags the amplitude recurrence (bit 2) but not
    the row pairs (bit 1), so the sweep's general row-pair instantiation (or, for the
    default row triples, their direct instantiation) runs; scores match the oracle's."""
    import torch
    system, D, _ = W.sweep_optics()
    det = W.Detector(128, 128, 4e-6, 4e-6)
    sw = W.Sweep(system, D, det, (16, 32, 64), (2.0, 3.0, 1.5), (1.0, 1.0, 1.2))
    flags = 0
    for k in range(sw.n_instances):
        b = gbd.trace(sw.system, sw.pupil(k))
        n = b.shape[0]
        coef = torch.empty(gbd.gbd_project_bytes(n, gbd.GBD_PREC_MIXED), dtype=torch.uint8,
                           device="cuda")
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
        gbd.gbd_project(b, n, sw.system.wavelength, det, gbd.GBD_PREC_MIXED, coef, flag)
        gbd.gbd_sync()
        flags |= int(flag.item())
    assert flags & 4 and not flags & 2, flags
    got = gbd.sweep_plan(sw, shape=shape).run().cpu().numpy()
    gbd.gbd_sync()
    want = oracle_scores(sw, range(sw.n_instances))
    assert np.max(np.abs(got - want)) <= SCORE_TOL, (got, want)
