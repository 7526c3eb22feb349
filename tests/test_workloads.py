"""The seeded synthetic inputs against the configurations they stand in for (host only):
optics, beamlet counts, detector spans in lambda F#, tilts, the Zernike draw, the sweep's
distributions and the parameter-search grid."""
import math

import numpy as np
import pytest

from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import workloads as W


def _half_span_lfd(wl):
    det = wl.detector
    lfd = wl.system.wavelength * wl.f_number
    return det.nx * det.pitch_x / 2.0 / lfd, det.ny * det.pitch_y / 2.0 / lfd


@pytest.mark.parametrize("name,lam,fnum,n_across,count,npix,span,of,wr", [
    ("airy_small", 1.0e-6, 10.0, 32, 812, 128, 5.0, 1.5, 1.5),
    ("airy_large", 1.0e-6, 10.0, 256, 51468, 512, 20.0, 1.5, 1.5),
    ("tilted_zernike", 0.633e-6, 5.0, 128, 12892, 1024, 15.0, 2.0, 1.2),
])
def test_field_workloads(name, lam, fnum, n_across, count, npix, span, of, wr):
    wl = W.by_name(name)
    assert wl.system.wavelength == lam and wl.pupil.diameter == 2.4e-3
    assert wl.f_number == pytest.approx(fnum)
    assert wl.system.distance == wl.system.focal_length  # the focal plane
    assert (wl.pupil.n_across, wl.pupil.overlap_factor, wl.pupil.waist_ratio) == (n_across, of, wr)
    assert gbd.gbd_beamlet_count(wl.pupil) == count
    assert (wl.detector.nx, wl.detector.ny) == (npix, npix)
    assert _half_span_lfd(wl) == pytest.approx((span, span))


def test_tilted_zernike_plate_and_tilt():
    wl = W.tilted_zernike()
    assert wl.system.noll == tuple(range(4, 16))
    assert wl.system.zern_radius == wl.pupil.diameter / 2
    # N(0, (0.05 lambda)^2) with the fixed seed, reproducible
    assert wl.system.zern_coef == W.zernike_draw(wl.system.wavelength, wl.system.noll)
    c = np.asarray(wl.system.zern_coef) / wl.system.wavelength
    assert np.all(np.abs(c) < 0.25) and 0.01 < np.std(c) < 0.1
    assert math.degrees(wl.detector.rot_x) == pytest.approx(10.0)
    assert math.degrees(wl.detector.rot_y) == pytest.approx(5.0)
    # the oracle's 64 x 64 strided subset
    cols, rows = W.strided_pixels(wl)
    assert cols.size == 64 and rows.size == 64


def test_sweep_distributions():
    sw = W.sweep()
    assert sw.n_instances == 1024
    assert (sw.detector.nx, sw.detector.ny) == (256, 256)
    n = np.asarray(sw.n_across)
    of = np.asarray(sw.overlap_factor)
    wr = np.asarray(sw.waist_ratio)
    assert set(np.unique(n)) == set(W.SWEEP_N_ACROSS)
    assert of.min() >= 1.0 and of.max() <= 3.0 and wr.min() >= 0.8 and wr.max() <= 3.0
    assert abs(of.mean() - 2.0) < 0.1 and abs(wr.mean() - 1.9) < 0.1
    counts = np.bincount([W.SWEEP_N_ACROSS.index(v) for v in n], minlength=5)
    assert counts.min() > 150  # each beamlet count about a fifth of the instances
    # reproducible from its seed
    assert W.sweep().n_across == sw.n_across


def test_search_grid():
    g = W.grid_sweep()
    assert g.n_instances == 1260
    assert len(set(g.overlap_factor)) == 21 and len(set(g.waist_ratio)) == 12
    assert set(g.n_across) == set(W.SWEEP_N_ACROSS)
    assert min(g.overlap_factor) == 1.0 and max(g.overlap_factor) == 3.0
    assert min(g.waist_ratio) == pytest.approx(0.8) and max(g.waist_ratio) == pytest.approx(3.0)


def test_telescope_sweep_refocus_is_the_least_rms_focus():
    """The telescope sweep's image plane sits midway between the real system's paraxial and
    marginal foci (the least-RMS-wavefront focus of third-order spherical aberration), from
    the oracle's real rays through the App. B prescription as printed."""
    import oracle
    msys, _, _ = W.hst_rc()

    def crossing(h):
        x, _, tx, _, _ = oracle.mirror_ray(msys, h, 0.0)
        return -x / tx  # axial distance from the printed image plane to the axis crossing

    paraxial, marginal = crossing(1e-3), crossing(0.5 * W.HST_DIAMETER[0])
    assert 100e-6 < paraxial < marginal < 120e-6
    assert W.HST_REFOCUS == pytest.approx(0.5 * (paraxial + marginal), abs=0.2e-6)
    msys2, D, F, det = W.telescope_optics()
    assert msys2.spacing[-1] == pytest.approx(W.HST_SPACING[-1] + W.HST_REFOCUS)
    assert D == W.HST_DIAMETER[0] and F == pytest.approx(24.0)
    assert (det.nx, det.ny) == (W.HST_SWEEP_NPIX, W.HST_SWEEP_NPIX)


def test_telescope_sweep_uses_the_seeded_draws():
    a, b = W.sweep(), W.telescope_sweep()
    assert (a.n_across, a.overlap_factor, a.waist_ratio) == (b.n_across, b.overlap_factor,
                                                             b.waist_ratio)
    sub = W.sweep_subset(b, [3, 1])
    assert isinstance(sub, W.MirrorSweep) and sub.n_across == (b.n_across[3], b.n_across[1])
    g = W.telescope_grid_sweep()
    assert g.n_instances == 1260 and g.system == b.system
