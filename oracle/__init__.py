"""FP64 CPU oracle of plane-evaluation Gaussian beamlet decomposition.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` may import this package.  It shares no code with
the CUDA library and the library never imports it.

The arithmetic lives in ``gbd_oracle.c`` (plain C, double precision, OpenMP over
pixels); this module marshals arguments, except for the truncated beamlets' edge factor
1/2 erfc(zeta) (``truncation_factor``), written here in numpy with scipy's complex erfc.  Inputs are duck-typed objects with the
attributes of the workload descriptions (``wavelength``, ``focal_length``, ...).

Pins (tests/test_oracle_pins.py): closed-form Gaussian beam, focal-plane structure-factor
identity, exact Airy peak and the Airy limit, direct Fresnel quadrature, energy
conservation, mirror symmetry, symplecticity, tilt = 0 reduction.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence, Tuple

import numpy as np
from scipy.special import erfc

from . import build as _build

REC_SIZE = 40
REC_RJ, REC_A, REC_W0, REC_ABCD, REC_P, REC_ALPHA, REC_L, REC_RHO, REC_THETA = (
    0, 2, 3, 4, 20, 28, 30, 31, 33)

_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_count.argtypes = [_I]
        L.orc_count.restype = _I
        L.orc_threads.restype = _I
        L.orc_trace.argtypes = [_D, _D, _D, _I, _PI, _PD, _D, _D, _I, _D, _D, _PD, _I]
        L.orc_trace.restype = _I
        L.orc_trace_truncated.argtypes = [_D, _D, _D, _I, _PI, _PD, _D, _D, _I, _D, _D, _D, _PD,
                                          _PD, _I, _PI]
        L.orc_trace_truncated.restype = _I
        for name in ("orc_field", "orc_field_exact"):
            fn = getattr(L, name)
            fn.argtypes = [_PD, _I, _D, _D, _D, _D, _I, _I, _D, _D, _PI, _I, _PI, _I, _PD]
            fn.restype = None
        L.orc_zernike.argtypes = [_I, _D, _D, _D, _PD, _PD, _PD]
        L.orc_noll.argtypes = [_I, _PI, _PI, _PI]
        L.orc_sqrtdet_v.argtypes = [_PD, _PD]
        L.orc_airy_amp.argtypes = [_D, _D, _D]
        L.orc_airy_amp.restype = _D
        L.orc_airy_score.argtypes = [_PD, _I, _I, _D, _D, _D, _D]
        L.orc_airy_score.restype = _D
        L.orc_zone_score.argtypes = [_PD, _I, _I, _D, _D, _D, _D, _D, _D]
        L.orc_zone_score.restype = _D
        L.orc_mirror_ray.argtypes = [_I, _PD, _PD, _PD, _D, _D, _D, _D, _D, _PD]
        L.orc_trace_mirrors.argtypes = [_D, _I, _PD, _PD, _PD, _D, _D, _I, _D, _D, _PD, _I]
        L.orc_trace_mirrors.restype = _I
        _lib = L
    return _lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _pi(a: np.ndarray):
    return a.ctypes.data_as(_PI)


def threads() -> int:
    return lib().orc_threads()


def count(n_across: int) -> int:
    """Number of beamlet centres inside the pupil for n_across beamlets across."""
    return lib().orc_count(int(n_across))


def trace(system, pupil) -> np.ndarray:
    """Beamlet table (n_b x 40 doubles), one row per beamlet in grid order."""
    nb = count(pupil.n_across)
    out = np.zeros((max(nb, 1), REC_SIZE), dtype=np.float64)
    noll = np.ascontiguousarray(np.asarray(system.noll, dtype=np.int32).reshape(-1))
    zc = np.ascontiguousarray(np.asarray(system.zern_coef, dtype=np.float64).reshape(-1))
    if noll.size == 0:
        noll = np.zeros(1, np.int32)
        zc = np.zeros(1, np.float64)
        nz = 0
    else:
        nz = int(noll.size)
    n = lib().orc_trace(system.wavelength, system.focal_length, system.distance, nz, _pi(noll),
                        _pd(zc), float(system.zern_radius), pupil.diameter, pupil.n_across,
                        pupil.overlap_factor, pupil.waist_ratio, _pd(out), out.shape[0])
    if n != nb:
        raise RuntimeError(f"oracle trace produced {n} beamlets, expected {nb}")
    return out[:nb]


def _pixels(detector, cols, rows):
    if cols is None:
        cols = np.arange(detector.nx)
    if rows is None:
        rows = np.arange(detector.ny)
    return (np.ascontiguousarray(np.asarray(cols, dtype=np.int32)),
            np.ascontiguousarray(np.asarray(rows, dtype=np.int32)))


def field(beamlets: np.ndarray, system, detector, cols: Optional[Sequence[int]] = None,
          rows: Optional[Sequence[int]] = None, exact: bool = False) -> np.ndarray:
    """Coherent beamlet sum at pixels (cols x rows); complex128 array [len(rows), len(cols)].

    ``exact`` evaluates each beamlet propagated exactly (paraxially) to every pixel's
    axial offset instead of the second-order plane rule (identical when untilted)."""
    b = np.ascontiguousarray(beamlets, dtype=np.float64)
    c, r = _pixels(detector, cols, rows)
    out = np.zeros((r.size, c.size, 2), dtype=np.float64)
    fn = lib().orc_field_exact if exact else lib().orc_field
    if b.shape[0] == 0:
        return np.zeros((r.size, c.size), dtype=np.complex128)
    fn(_pd(b), b.shape[0], system.wavelength, getattr(system, "distance", 0.0), detector.rot_x,
       detector.rot_y,
       detector.nx, detector.ny, detector.pitch_x, detector.pitch_y, _pi(c), c.size, _pi(r),
       r.size, _pd(out))
    return out[..., 0] + 1j * out[..., 1]


def trace_truncated(system, pupil, margin: float = 3.0):
    """Truncated decomposition (edge beamlets cut by the aperture's tangent half-plane):
    (records, dist, n_edge), interior beamlets first, then edge beamlets; dist holds each
    edge beamlet's signed distance d_j = R - |r_j| to the edge and +inf for interior ones."""
    N = pupil.n_across
    cap = (N + 2 * (int(math.ceil(0.5 * margin * pupil.overlap_factor)) + 1)) ** 2
    out = np.zeros((cap, REC_SIZE), dtype=np.float64)
    dist = np.zeros(cap, dtype=np.float64)
    noll = np.ascontiguousarray(np.asarray(system.noll, dtype=np.int32).reshape(-1))
    zc = np.ascontiguousarray(np.asarray(system.zern_coef, dtype=np.float64).reshape(-1))
    nz = int(noll.size)
    if nz == 0:
        noll = np.zeros(1, dtype=np.int32)
        zc = np.zeros(1)
    ne = _I()
    n = lib().orc_trace_truncated(system.wavelength, system.focal_length, system.distance, nz,
                                  _pi(noll), _pd(zc), float(system.zern_radius),
                                  pupil.diameter, N, pupil.overlap_factor, pupil.waist_ratio,
                                  float(margin), _pd(out), _pd(dist), cap, ctypes.byref(ne))
    if n < 0:
        raise RuntimeError("oracle truncated trace: capacity too small")
    return out[:n], dist[:n], int(ne.value)


def truncation_factor(rec: np.ndarray, normal, d: float, wavelength: float, X, Y) -> np.ndarray:
    """1/2 erfc(zeta) that turns beamlet `rec`'s Gaussian into the field of its input cut by
    the half-plane n.(r - r_j) <= d (the Collins integral of Eq. collins over that half-plane
    divided by the full one), at lab points (X, Y) of the untilted reference plane:
        M = A + B P1,  zeta = (n^T M^-1 (rho - rho_c) - d) sqrt(i k / (2 n^T M^-1 B n)),
    principal square root (its real part > 0 keeps the cut Gaussian integrable)."""
    k = 2.0 * math.pi / wavelength
    w0 = rec[REC_W0]
    A = rec[REC_ABCD:REC_ABCD + 4].reshape(2, 2)
    B = rec[REC_ABCD + 4:REC_ABCD + 8].reshape(2, 2)
    M = A + B * (-1j * wavelength / (math.pi * w0 * w0))
    Mi = np.linalg.inv(M)
    n = np.asarray(normal, dtype=np.float64)
    sigma = n @ Mi @ B @ n
    root = np.sqrt(1j * k / (2.0 * sigma))
    u = n @ Mi  # row vector n^T M^-1
    t = u[0] * (X - rec[REC_RHO]) + u[1] * (Y - rec[REC_RHO + 1])
    return 0.5 * erfc((t - d) * root)


def field_truncated(records: np.ndarray, dist: np.ndarray, system, detector,
                    cols: Optional[Sequence[int]] = None, rows: Optional[Sequence[int]] = None,
                    normals: Optional[np.ndarray] = None) -> np.ndarray:
    """Coherent sum of a truncated decomposition on an untilted detector: interior beamlets
    (dist = +inf) as Gaussians (orc_field), each edge beamlet's Gaussian times its truncation
    factor.  normals: per-beamlet edge normals (default r_j / |r_j|)."""
    if detector.rot_x != 0.0 or detector.rot_y != 0.0:
        raise ValueError("truncated beamlets are evaluated on untilted planes")
    c, r = _pixels(detector, cols, rows)
    inner = ~np.isfinite(dist)
    E = field(records[inner], system, detector, c, r) if inner.any() else \
        np.zeros((r.size, c.size), dtype=np.complex128)
    X = ((c - detector.nx // 2) * detector.pitch_x)[None, :]
    Y = ((r - detector.ny // 2) * detector.pitch_y)[:, None]
    for q in np.flatnonzero(~inner):
        rec = records[q]
        nrm = normals[q] if normals is not None else rec[REC_RJ:REC_RJ + 2] / np.hypot(
            rec[REC_RJ], rec[REC_RJ + 1])
        g = field(rec[None, :], system, detector, c, r)
        E = E + g * truncation_factor(rec, nrm, dist[q], system.wavelength, X, Y)
    return E


def zernike(j: int, radius: float, x: float, y: float) -> Tuple[float, float, float]:
    """Noll mode j (RMS-normalised on the disk of ``radius``) and its gradient at (x, y)."""
    z, zx, zy = _D(), _D(), _D()
    lib().orc_zernike(int(j), radius, x, y, ctypes.byref(z), ctypes.byref(zx), ctypes.byref(zy))
    return z.value, zx.value, zy.value


def noll(j: int) -> Tuple[int, int, bool]:
    n, m, s = _I(), _I(), _I()
    lib().orc_noll(int(j), ctypes.byref(n), ctypes.byref(m), ctypes.byref(s))
    return n.value, m.value, bool(s.value)


def sqrtdet(m: np.ndarray) -> complex:
    """sqrt(det M) on the eigenvalue branch, for a 2x2 complex matrix."""
    a = np.asarray(m, dtype=np.complex128).reshape(2, 2)
    buf = np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1).reshape(-1))
    out = np.zeros(2)
    lib().orc_sqrtdet_v(_pd(buf), _pd(out))
    return complex(out[0], out[1])


def airy_amp(r: float, wavelength: float, f_number: float) -> float:
    return lib().orc_airy_amp(float(r), wavelength, f_number)


def airy_score(field_: np.ndarray, detector, wavelength: float, f_number: float) -> float:
    """RMS of |E|/|E(centre)| - |2 J1(x)/x| inside the third dark ring."""
    f = np.ascontiguousarray(np.stack([field_.real, field_.imag], axis=-1), dtype=np.float64)
    return lib().orc_airy_score(_pd(f), detector.nx, detector.ny, detector.pitch_x,
                                detector.pitch_y, wavelength, f_number)


def zone_score(field_: np.ndarray, detector, wavelength: float, f_number: float, lo: float,
               hi: float) -> float:
    """RMS of |E|/|E(centre)| - |2 J1(x)/x| over lo <= r/(lambda F#) < hi (Sec. 6 zones)."""
    f = np.ascontiguousarray(np.stack([field_.real, field_.imag], axis=-1), dtype=np.float64)
    return lib().orc_zone_score(_pd(f), detector.nx, detector.ny, detector.pitch_x,
                                detector.pitch_y, wavelength, f_number, lo, hi)


def _mirror_arrays(msys):
    n = len(msys.radius)
    return (n, np.ascontiguousarray(msys.radius, dtype=np.float64),
            np.ascontiguousarray(msys.conic, dtype=np.float64),
            np.ascontiguousarray(msys.spacing, dtype=np.float64))


def mirror_ray(msys, x0: float, y0: float, ax: float = 0.0, ay: float = 0.0) -> np.ndarray:
    """Real ray through the mirrors: (x, y, theta_x, theta_y, path) at the image plane."""
    n, R, K, T = _mirror_arrays(msys)
    out = np.zeros(5)
    lib().orc_mirror_ray(n, _pd(R), _pd(K), _pd(T), msys.pupil_offset, x0, y0, ax, ay, _pd(out))
    return out


def trace_mirrors(msys, pupil) -> np.ndarray:
    """Beamlet table of a pupil in front of a sequence of conic mirrors."""
    nb = count(pupil.n_across)
    out = np.zeros((max(nb, 1), REC_SIZE), dtype=np.float64)
    n, R, K, T = _mirror_arrays(msys)
    got = lib().orc_trace_mirrors(msys.wavelength, n, _pd(R), _pd(K), _pd(T), msys.pupil_offset,
                                  pupil.diameter, pupil.n_across, pupil.overlap_factor,
                                  pupil.waist_ratio, _pd(out), out.shape[0])
    if got != nb:
        raise RuntimeError(f"oracle mirror trace produced {got} beamlets, expected {nb}")
    return out[:nb]


def unpack(rec: np.ndarray) -> dict:
    """Named views of one beamlet record."""
    A = rec[REC_ABCD:REC_ABCD + 4].reshape(2, 2)
    B = rec[REC_ABCD + 4:REC_ABCD + 8].reshape(2, 2)
    C = rec[REC_ABCD + 8:REC_ABCD + 12].reshape(2, 2)
    D = rec[REC_ABCD + 12:REC_ABCD + 16].reshape(2, 2)
    P = (rec[REC_P:REC_P + 8:2] + 1j * rec[REC_P + 1:REC_P + 8:2]).reshape(2, 2)
    return dict(r=rec[REC_RJ:REC_RJ + 2], a=rec[REC_A], w0=rec[REC_W0], A=A, B=B, C=C, D=D,
                P=P, alpha=complex(rec[REC_ALPHA], rec[REC_ALPHA + 1]), L=rec[REC_L],
                rho=rec[REC_RHO:REC_RHO + 2], theta=rec[REC_THETA:REC_THETA + 2])
