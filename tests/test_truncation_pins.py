"""Pins of the oracle's truncated beamlets (edge beamlets cut by the aperture's tangent
half-plane; Sec. 1 and the Conclusion name Worku & Gross's truncated beamlets as the way to
represent hard aperture edges).

A Gaussian cut by a straight edge stays integrable in closed form through any paraxial
system: the Collins integral of Eq. collins over the half-plane equals the untruncated
beamlet times 1/2 erfc(zeta), zeta affine in the output coordinate.  The pins check that
factor against direct quadrature of the Fresnel integral (Eq. fresnel, the exp(-ik.)
convention of the other Fresnel pins) over the half-plane, its limits, the decomposition's
bookkeeping against brute force, and, for a hard circular aperture at the focal plane of a
thin lens, against the exact field (i / (lambda f)) e^(-ik r^2/2f) pi R^2 2 J1(x)/x.
"""
import math

import numpy as np
import pytest
from scipy.special import j1

import oracle
from paper_2404_12454_gb300 import workloads as W


def _k(lam):
    return 2.0 * math.pi / lam


def _fresnel_cut(ax, ay, rj, n, d, w0, f, z, lam, nq=2400, half=7.0):
    """Direct quadrature of the Fresnel integral of exp(-|r1 - rj|^2/w0^2) behind a thin lens
    of focal length f, cut to n.(r1 - rj) <= d, at output points (ax, ay) a distance z away
    (prefactor i/(lambda z); the axial phase is dropped).  In edge coordinates r1 = rj + t n
    + s m the integrand factorises into a t-integral over [-half w0, d] and an s-integral
    over [-half w0, half w0]."""
    k = _k(lam)
    m = np.array([-n[1], n[0]])
    c = 1.0 / f - 1.0 / z
    X = np.stack([ax, ay], axis=-1)  # output points (..., 2)
    xn, xm = X @ n, X @ m
    rn, rm = float(rj @ n), float(rj @ m)

    def line(lo, hi, r0, xc):
        t, w = np.polynomial.legendre.leggauss(nq)
        u = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
        wt = 0.5 * (hi - lo) * w
        ph = -(u / w0) ** 2 + 0.5j * k * c * (2.0 * r0 * u + u * u)
        return (np.exp(ph)[None, :] * np.exp(1j * k * np.outer(xc.ravel(), u) / z)) @ wt

    Ft = line(-half * w0, d, rn, xn).reshape(xn.shape)
    Fs = line(-half * w0, half * w0, rm, xm).reshape(xm.shape)
    const = np.exp(0.5j * k * c * float(rj @ rj) + 1j * k * (X @ rj) / z
                   - 0.5j * k * np.sum(X * X, axis=-1) / z)
    return (1j / (lam * z)) * const * Ft * Fs


@pytest.mark.parametrize("d_over_w0", [-0.8, 0.0, 0.5, 1.5])
@pytest.mark.parametrize("phi", [0.0, 0.7, 2.5])
def test_cut_beamlet_matches_fresnel_quadrature(d_over_w0, phi):
    """One beamlet of a 3 x 3 decomposition (centre (1 mm, 1 mm), w0 0.75 mm) behind an
    f = 50 mm lens, observed 52 mm away, cut by edges of three orientations at four
    offsets; the closed form matches quadrature to 1e-9 of the peak."""
    lam, f, z = 1e-6, 0.05, 0.052
    sysm = W.System(lam, f, z)
    b = oracle.trace(sysm, W.Pupil(3e-3, 3, 1.5, 1.0))
    rec = b[2 * 3 + 2]
    u = oracle.unpack(rec)
    assert np.allclose(u["r"], [1e-3, 1e-3])
    w0 = u["w0"]
    n = np.array([math.cos(phi), math.sin(phi)])
    d = d_over_w0 * w0
    p = 4e-6
    det = W.Detector(64, 64, p, p)
    cols = rows = np.arange(20, 44, 2)  # around the chief ray's landing, (1 - z/f) r_j
    G = oracle.field(rec[None, :], sysm, det, cols, rows)
    X = ((cols - 32) * p)[None, :] * np.ones((rows.size, 1))
    Y = ((rows - 32) * p)[:, None] * np.ones((1, cols.size))
    E = G * oracle.truncation_factor(rec, n, d, lam, X, Y)
    Et = u["a"] * _fresnel_cut(X, Y, u["r"], n, d, w0, f, z, lam)
    scale = np.max(np.abs(u["a"] * _fresnel_cut(X, Y, u["r"], n, 12 * w0, w0, f, z, lam)))
    assert np.max(np.abs(E - Et)) < 1e-9 * scale, np.max(np.abs(E - Et)) / scale


def test_cut_factor_limits():
    """An edge far outside the beamlet leaves it whole (factor 1); an edge far inside the
    other way removes it (factor 0); an edge through the beamlet's centre gives exactly 1/2
    at the chief ray's landing (zeta = 0 there)."""
    lam, f = 1e-6, 0.05
    sysm = W.System(lam, f, f)
    rec = oracle.trace(sysm, W.Pupil(3e-3, 3, 1.5, 1.0))[4]  # the centre beamlet
    w0 = rec[oracle.REC_W0]
    x = np.linspace(-40e-6, 40e-6, 9)
    X, Y = np.meshgrid(x, x)
    n = np.array([0.6, 0.8])
    one = oracle.truncation_factor(rec, n, 12 * w0, lam, X, Y)
    zero = oracle.truncation_factor(rec, n, -12 * w0, lam, X, Y)
    assert np.max(np.abs(one - 1.0)) < 1e-14 and np.max(np.abs(zero)) < 1e-14
    half = oracle.truncation_factor(rec, n, 0.0, lam, np.zeros(1), np.zeros(1))
    assert abs(half[0] - 0.5) < 1e-15


def test_truncated_decomposition_bookkeeping():
    """Centres out to R + 3 w0, interior ones (more than 3 w0 inside) first, then the edge
    ones, each in row-major grid order; d_j = R - |r_j|; the weights and waists are those
    of the plain decomposition, whose beamlets are all among these."""
    wl = W.airy_small()
    D, N, OF = wl.pupil.diameter, wl.pupil.n_across, wl.pupil.overlap_factor
    recs, dist, n_edge = oracle.trace_truncated(wl.system, wl.pupil, margin=3.0)
    s, w0, R = D / N, OF * D / (2 * N), D / 2
    want_in, want_edge = [], []
    for j in range(-10, N + 10):
        for i in range(-10, N + 10):
            x, y = (i - (N - 1) / 2) * s, (j - (N - 1) / 2) * s
            rr = math.hypot(x, y)
            if rr > R + 3 * w0 + 1e-12:
                continue
            (want_in if rr < R - 3 * w0 - 1e-12 else want_edge).append((x, y, R - rr))
    assert n_edge == len(want_edge) and recs.shape[0] == len(want_in) + len(want_edge)
    got = recs[:, oracle.REC_RJ:oracle.REC_RJ + 2]
    assert np.allclose(got[:len(want_in)], np.array(want_in)[:, :2], rtol=0, atol=1e-15)
    assert np.allclose(got[len(want_in):], np.array(want_edge)[:, :2], rtol=0, atol=1e-15)
    assert np.all(np.isinf(dist[:len(want_in)]))
    assert np.allclose(dist[len(want_in):], np.array(want_edge)[:, 2], rtol=0, atol=1e-15)
    assert np.all(recs[:, oracle.REC_W0] == w0)
    assert np.allclose(recs[:, oracle.REC_A], s * s / (math.pi * w0 * w0), rtol=1e-15)
    plain = oracle.trace(wl.system, wl.pupil)
    keys = {(round(a / s * 2), round(b / s * 2)) for a, b in got}
    assert all((round(a / s * 2), round(b / s * 2)) in keys
               for a, b in plain[:, oracle.REC_RJ:oracle.REC_RJ + 2])


def test_zero_margin_is_the_plain_decomposition():
    """With no margin no centre of an even grid lies on the edge circle, so every beamlet
    is interior and the field is the plain decomposition's."""
    wl = W.scaled(W.airy_small(), n_across=20, nx=40, ny=40)
    recs, dist, n_edge = oracle.trace_truncated(wl.system, wl.pupil, margin=0.0)
    assert n_edge == 0 and recs.shape[0] == oracle.count(20)
    E0 = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    E1 = oracle.field_truncated(recs, dist, wl.system, wl.detector)
    assert np.array_equal(E0, E1)


def _exact_focal_field(wl):
    """Uniform circular aperture behind an ideal lens, at its focal plane (Fraunhofer, Eq.
    fraunhofer): (i / (lambda f)) e^(-ik r^2/2f) pi R^2 2 J1(x)/x, x = k R r / f."""
    lam, f, R = wl.system.wavelength, wl.system.focal_length, wl.pupil.diameter / 2
    det = wl.detector
    k = _k(lam)
    x = (np.arange(det.nx) - det.nx // 2) * det.pitch_x
    y = (np.arange(det.ny) - det.ny // 2) * det.pitch_y
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    u = k * R * r / f
    safe = np.where(u == 0, 1.0, u)
    airy = np.where(u == 0, 1.0, 2 * j1(safe) / safe)
    return (1j / (lam * f)) * np.exp(-1j * k * r * r / (2 * f)) * math.pi * R * R * airy


def test_truncated_beamlets_reproduce_the_hard_aperture():
    """On the small Airy workload's optics and detector (32 across, OF 1.5) the truncated
    decomposition's field is 10x closer to the exact hard-aperture field than the plain
    one's (measured 1.9e-3 against 2.6e-2 relative L2), and its error falls with N."""
    wl = W.airy_small()
    exact = _exact_focal_field(wl)

    def err(E):
        return np.linalg.norm(E - exact) / np.linalg.norm(exact)

    plain = err(oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector))
    recs, dist, _ = oracle.trace_truncated(wl.system, wl.pupil)
    cut = err(oracle.field_truncated(recs, dist, wl.system, wl.detector))
    assert cut < 3e-3 and cut < 0.1 * plain, (cut, plain)
    errs = []
    for N in (16, 32, 48):
        w = W.scaled(wl, n_across=N)
        recs, dist, _ = oracle.trace_truncated(w.system, w.pupil)
        errs.append(err(oracle.field_truncated(recs, dist, w.system, w.detector)))
    assert errs[0] > errs[1] > errs[2], errs
