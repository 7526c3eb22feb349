"""Truncated beamlets on the GPU (gbd_trace_truncated, gbd_field_truncated) against the
oracle's truncated decomposition: records field by field, fields to 1e-11 (FP64) and 2e-5
(mixed) relative L2, and the gain of the cut beamlets against the exact hard-aperture field
at the focal plane of a thin lens."""
import math

import numpy as np
import pytest
from scipy.special import j1

import oracle
from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {gbd.GBD_PREC_F64: 1e-11, gbd.GBD_PREC_MIXED: 2e-5}
PRECS = (gbd.GBD_PREC_F64, gbd.GBD_PREC_MIXED)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_12454_gb300 import build
    build.build()
    import torch
    torch.cuda.init()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cases():
    airy = W.airy_small()
    tz = W.tilted_zernike()
    untilted_tz = W.Workload("zernike_untilted", tz.system, W.Pupil(2.4e-3, 20, 2.0, 1.2),
                             W.Detector(72, 56, 0.35e-6, 0.4e-6))
    return {
        "airy_small": airy,
        "airy_ragged": W.scaled(airy, n_across=23, nx=97, ny=45),
        "defocused": W.Workload("defocused", W.System(1e-6, 0.024, 0.0246),
                                W.Pupil(2.4e-3, 16, 1.2, 2.0), W.Detector(70, 66, 1.5e-6, 1.2e-6)),
        "zernike_untilted": untilted_tz,
        "all_edge": W.Workload("all_edge", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 4, 1.5, 1.0),
                               W.Detector(40, 40, 2e-6, 2e-6)),
    }


@pytest.mark.parametrize("name", list(cases()))
def test_truncated_records_match_oracle(name):
    wl = cases()[name]
    b, ne = gbd.trace_truncated(wl.system, wl.pupil)
    gbd.gbd_sync()
    o, dist, one = oracle.trace_truncated(wl.system, wl.pupil)
    assert b.shape[0] == o.shape[0] and ne == one
    g = b.cpu().numpy()
    for k, (rg, ro) in enumerate(zip(g, o)):
        a, c = gbd.unpack(rg), oracle.unpack(ro)
        assert np.allclose(a["center"], c["r"], rtol=0, atol=1e-18)
        if np.isfinite(dist[k]):
            assert abs(a["edge_distance"] - dist[k]) <= 1e-18
        else:
            assert a["edge_distance"] == 0.0
        assert abs(a["weight"] - c["a"]) <= 1e-15 * c["a"]
        assert np.allclose(a["rho"], c["rho"], rtol=0, atol=1e-16)
        assert np.allclose(a["theta"], c["theta"], rtol=0, atol=1e-14)
        assert np.allclose(a["P"], c["P"], rtol=0, atol=1e-10 * np.abs(c["P"]).max())
        assert abs(a["amp"] - c["alpha"]) <= 1e-12 * abs(c["alpha"])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(cases()))
def test_truncated_field_matches_oracle(name, prec):
    wl = cases()[name]
    b, ne = gbd.trace_truncated(wl.system, wl.pupil)
    E = gbd.field_truncated(b, ne, wl.system.wavelength, wl.detector, prec)
    gbd.gbd_sync()
    o, dist, _ = oracle.trace_truncated(wl.system, wl.pupil)
    Eo = oracle.field_truncated(o, dist, wl.system, wl.detector)
    err = rel_l2(E.cpu().numpy().astype(np.complex128), Eo)
    assert err <= TOL[prec], err


def exact_focal_field(wl):
    lam, f, R = wl.system.wavelength, wl.system.focal_length, wl.pupil.diameter / 2
    det = wl.detector
    k = 2 * math.pi / lam
    x = (np.arange(det.nx) - det.nx // 2) * det.pitch_x
    y = (np.arange(det.ny) - det.ny // 2) * det.pitch_y
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    u = k * R * r / f
    safe = np.where(u == 0, 1.0, u)
    airy = np.where(u == 0, 1.0, 2 * j1(safe) / safe)
    return (1j / (lam * f)) * np.exp(-1j * k * r * r / (2 * f)) * math.pi * R * R * airy


@pytest.mark.parametrize("prec", PRECS)
def test_truncated_beamlets_cut_the_edge_error_on_the_small_airy_workload(prec):
    """32 across, OF 1.5, 128^2 pixels over +-5 lambda F#: the field's distance to the exact
    hard-aperture focal field drops from 2.6e-2 (plain decomposition, gbd_field) to 1.9e-3
    (truncated, gbd_field_truncated), on the GPU as in the oracle."""
    wl = W.airy_small()
    exact = exact_focal_field(wl)
    plain = gbd.field(gbd.trace(wl.system, wl.pupil), wl.system.wavelength, wl.detector, prec)
    b, ne = gbd.trace_truncated(wl.system, wl.pupil)
    cut = gbd.field_truncated(b, ne, wl.system.wavelength, wl.detector, prec)
    gbd.gbd_sync()
    e_plain = rel_l2(plain.cpu().numpy().astype(np.complex128), exact)
    e_cut = rel_l2(cut.cpu().numpy().astype(np.complex128), exact)
    assert e_cut < 3e-3 and e_cut < 0.1 * e_plain, (e_cut, e_plain)


def test_truncated_edge_cases():
    import torch
    wl = W.airy_small()
    # no margin: no edge beamlets, the plain decomposition's field bit for bit
    pupil = wl.pupil
    n, ne = gbd.gbd_truncated_count(pupil, pupil.overlap_factor, 0.0)
    assert ne == 0 and n == gbd.gbd_beamlet_count(pupil)
    b, ne = gbd.trace_truncated(wl.system, pupil, margin=0.0)
    E0 = gbd.field(gbd.trace(wl.system, pupil), wl.system.wavelength, wl.detector,
                   gbd.GBD_PREC_MIXED)
    E1 = gbd.field_truncated(b, 0, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED)
    gbd.gbd_sync()
    assert torch.equal(E0, E1)
    b, ne = gbd.trace_truncated(wl.system, pupil)
    out = torch.empty((wl.detector.ny, wl.detector.nx), dtype=torch.complex64, device="cuda")
    ws = torch.empty(gbd.gbd_field_truncated_workspace_bytes(b.shape[0], ne, wl.detector,
                                                             gbd.GBD_PREC_MIXED),
                     dtype=torch.uint8, device="cuda")
    tilted = W.Detector(wl.detector.nx, wl.detector.ny, wl.detector.pitch_x, wl.detector.pitch_y,
                        0.1, 0.0)
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_field_truncated(b, b.shape[0], ne, wl.system.wavelength, tilted,
                                gbd.GBD_PREC_MIXED, ws, out)
    assert ei.value.status == gbd.GBD_EUNSUPPORTED
    with pytest.raises(gbd.GbdError):
        gbd.gbd_field_truncated(b, b.shape[0], b.shape[0] + 1, wl.system.wavelength,
                                wl.detector, gbd.GBD_PREC_MIXED, ws, out)
    small = torch.empty((1, 36), dtype=torch.float64, device="cuda")
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_trace_truncated(wl.system, pupil, pupil.overlap_factor, pupil.waist_ratio, 3.0,
                                small)
    assert ei.value.status == gbd.GBD_ENOMEM


@pytest.mark.parametrize("prec", PRECS)
def test_truncated_field_is_deterministic_and_split_sized(prec):
    """The edge beamlets are split over CTAs into partial fields added in split order: two
    evaluations give the same bits; a detector of 333 x 7 pixels (ragged 8-pixel row
    segments, many splits per pixel block) still matches the oracle."""
    wl = W.scaled(W.airy_small(), nx=333, ny=7)
    b, ne = gbd.trace_truncated(wl.system, wl.pupil)
    E1 = gbd.field_truncated(b, ne, wl.system.wavelength, wl.detector, prec)
    E2 = gbd.field_truncated(b, ne, wl.system.wavelength, wl.detector, prec)
    gbd.gbd_sync()
    assert np.array_equal(E1.cpu().numpy(), E2.cpu().numpy())
    o, dist, _ = oracle.trace_truncated(wl.system, wl.pupil)
    Eo = oracle.field_truncated(o, dist, wl.system, wl.detector)
    err = rel_l2(E1.cpu().numpy().astype(np.complex128), Eo)
    assert err <= TOL[prec], err
