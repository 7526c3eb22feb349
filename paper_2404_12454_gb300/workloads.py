"""Seeded synthetic workloads for plane-evaluation Gaussian beamlet decomposition.

This module only *describes inputs*: optical prescriptions, pupil sampling, detector
geometry, random draws and sizes.  It holds none of the method's arithmetic, so both
the CUDA library's callers and the FP64 CPU oracle's tests build their inputs from it.

The paper's experiments use a Zemax-traced Hubble-like telescope (Sec. 4.2, App. B)
whose ray data is not public.  Paraxial GBD expressed in units of lambda*F/# is
scale-free, so an ideal thin lens of the same focal ratio per lambda*F/# stands in
for it: the beamlet envelope at focus is w_f = lambda*f/(pi*w0) = (2N/(pi*OF)) *
lambda*F/#, independent of the absolute pupil size (Eq. OF, Sec. 6).

Five workloads:

* ``airy_small``   -- 2.4 mm pupil, lambda 1 um, F/10 lens focused on its focal
  plane, 32 beamlets across (812 inside), OF 1.5, 128x128 pixels over +-5 lambda F/#.
* ``airy_large``   -- same optics, 256 across (51,468 beamlets), 512x512 over
  +-20 lambda F/#.
* ``tilted_zernike`` -- F/5, lambda 0.633 um, Noll Z4..Z15 OPD plate drawn from
  N(0, (0.05 lambda)^2), 128 across (12,892 beamlets), OF 2.0, waist ratio 1.2,
  1024x1024 pixels over +-15 lambda F/#, detector tilted 10 deg about x, 5 deg about y.
* ``sweep``        -- 1024 instances of the airy_small optics with OF ~ U[1,3],
  waist ratio ~ U[0.8,3], beamlets across ~ U{16,32,64,128,256}, 256x256 pixels
  over +-5 lambda F/#.
* ``surrogate``    -- the MLP search over the sweep's parameter space.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_ZERNIKE = 240412454
SEED_SWEEP = 240412455
SEED_SURROGATE = 240412456

# Number of beamlets across the pupil that the parameter search may use (Sec. 6).
SWEEP_N_ACROSS = (16, 32, 64, 128, 256)


@dataclasses.dataclass(frozen=True)
class System:
    """Paraxial system: optional Zernike OPD plate at the pupil, thin lens f, distance d.

    ``noll`` / ``zern_coef`` are Noll indices and RMS-normalised coefficients in metres
    of optical path over the disk of radius ``zern_radius``.
    """

    wavelength: float
    focal_length: float
    distance: float
    noll: Tuple[int, ...] = ()
    zern_coef: Tuple[float, ...] = ()
    zern_radius: float = 1.0


@dataclasses.dataclass(frozen=True)
class Pupil:
    """Uniform circular pupil of ``diameter`` sampled by ``n_across`` beamlets across."""

    diameter: float
    n_across: int
    overlap_factor: float
    waist_ratio: float


@dataclasses.dataclass(frozen=True)
class Detector:
    """Pixel grid on a plane through (0, 0, d) rotated by R = Ry(rot_y) Rx(rot_x).

    Pixel (i, j) (column i along x, row j along y) sits at detector coordinates
    s = ((i - nx//2) * pitch_x, (j - ny//2) * pitch_y), so a pixel lies on the axis.
    """

    nx: int
    ny: int
    pitch_x: float
    pitch_y: float
    rot_x: float = 0.0
    rot_y: float = 0.0


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    system: System
    pupil: Pupil
    detector: Detector
    # strided pixel subset on which the oracle is evaluated (None = every pixel)
    oracle_stride: Optional[Tuple[int, int]] = None  # (offset, step) on both axes

    @property
    def f_number(self) -> float:
        return self.system.focal_length / self.pupil.diameter


def _span_pitch(n: int, half_span_lfd: float, wavelength: float, f_number: float) -> float:
    """Pixel pitch for n pixels spanning +-half_span_lfd lambda*F/#."""
    return 2.0 * half_span_lfd * wavelength * f_number / n


def airy_small() -> Workload:
    lam, D, f = 1.0e-6, 2.4e-3, 24.0e-3
    p = _span_pitch(128, 5.0, lam, f / D)
    return Workload(
        "airy_small",
        System(lam, f, f),
        Pupil(D, 32, 1.5, 1.5),
        Detector(128, 128, p, p),
    )


def airy_large() -> Workload:
    lam, D, f = 1.0e-6, 2.4e-3, 24.0e-3
    p = _span_pitch(512, 20.0, lam, f / D)
    return Workload(
        "airy_large",
        System(lam, f, f),
        Pupil(D, 256, 1.5, 1.5),
        Detector(512, 512, p, p),
    )


def zernike_draw(wavelength: float, noll: Sequence[int] = tuple(range(4, 16)),
                 sigma_waves: float = 0.05, seed: int = SEED_ZERNIKE) -> Tuple[float, ...]:
    """Coefficients c_j ~ N(0, (sigma_waves*lambda)^2), in metres, one per Noll index."""
    rng = np.random.default_rng(seed)
    return tuple(float(v) for v in rng.normal(0.0, sigma_waves * wavelength, size=len(noll)))


def tilted_zernike() -> Workload:
    lam, D, f = 0.633e-6, 2.4e-3, 12.0e-3
    noll = tuple(range(4, 16))
    coef = zernike_draw(lam, noll)
    p = _span_pitch(1024, 15.0, lam, f / D)
    return Workload(
        "tilted_zernike",
        System(lam, f, f, noll, coef, D / 2.0),
        Pupil(D, 128, 2.0, 1.2),
        Detector(1024, 1024, p, p, math.radians(10.0), math.radians(5.0)),
        oracle_stride=(8, 16),
    )


@dataclasses.dataclass(frozen=True)
class Sweep:
    """A batch of GBD instances sharing optics and detector, differing in (N, OF, WR)."""

    system: System
    diameter: float
    detector: Detector
    n_across: Tuple[int, ...]
    overlap_factor: Tuple[float, ...]
    waist_ratio: Tuple[float, ...]

    @property
    def n_instances(self) -> int:
        return len(self.n_across)

    def pupil(self, k: int) -> Pupil:
        return Pupil(self.diameter, self.n_across[k], self.overlap_factor[k], self.waist_ratio[k])


def sweep_optics() -> Tuple[System, float, Detector]:
    lam, D, f = 1.0e-6, 2.4e-3, 24.0e-3
    p = _span_pitch(256, 5.0, lam, f / D)
    return System(lam, f, f), D, Detector(256, 256, p, p)


def sweep(n_instances: int = 1024, seed: int = SEED_SWEEP) -> Sweep:
    system, D, det = sweep_optics()
    rng = np.random.default_rng(seed)
    of = rng.uniform(1.0, 3.0, size=n_instances)
    wr = rng.uniform(0.8, 3.0, size=n_instances)
    n = rng.choice(np.asarray(SWEEP_N_ACROSS), size=n_instances)
    return Sweep(system, D, det, tuple(int(v) for v in n), tuple(float(v) for v in of),
                 tuple(float(v) for v in wr))


def grid_sweep() -> Sweep:
    """The regular reference grid of the parameter search: 21 OF x 12 WR x 5 N = 1,260."""
    system, D, det = sweep_optics()
    ofs = np.linspace(1.0, 3.0, 21)
    wrs = np.linspace(0.8, 3.0, 12)
    n, of, wr = [], [], []
    for N in SWEEP_N_ACROSS:
        for a in ofs:
            for b in wrs:
                n.append(int(N)), of.append(float(a)), wr.append(float(b))
    return Sweep(system, D, det, tuple(n), tuple(of), tuple(wr))


# Annular zones of Sec. 6, in lambda/D (= lambda F# on the focal plane).
ANNULAR_ZONES = ((0.0, 5.0), (5.0, 10.0), (10.0, 15.0))


def zone_sweep(of_values: Sequence[float] = tuple(np.linspace(1.0, 2.0, 11)),
               n_across: Sequence[int] = (32, 64, 128, 256), waist_ratio: float = 1.0) -> Sweep:
    """OF x N grid on the airy optics with a 512x512 detector over +-15.2 lambda F#: the
    paper's parameter-search sampling (App. D: 512^2 pixels of 2.8 mas, i.e. 0.059 lambda/D
    at lambda 551 nm, D 2.4 m) scaled to these optics, wide enough for the 10-15 lambda/D zone."""
    lam, D, f = 1.0e-6, 2.4e-3, 24.0e-3
    p = 0.0592 * lam * f / D
    det = Detector(512, 512, p, p)
    n, of, wr = [], [], []
    for N in n_across:
        for a in of_values:
            n.append(int(N)), of.append(float(a)), wr.append(float(waist_ratio))
    return Sweep(System(lam, f, f), D, det, tuple(n), tuple(of), tuple(wr))


@dataclasses.dataclass(frozen=True)
class MirrorSystem:
    """Sequence of reflective conic surfaces, light entering along +z, with App. B's sign
    for the radii (negative = concave, positive = convex towards the arriving light) and
    the signed axial distance from each vertex to the next surface (the last one: to the
    image plane).  The entrance pupil is a plane `pupil_offset` before the first vertex."""

    wavelength: float
    radius: Tuple[float, ...]
    conic: Tuple[float, ...]
    spacing: Tuple[float, ...]
    diameter: Tuple[float, ...]
    pupil_offset: float = 0.1


# App. B: Hubble-like Ritchey-Chretien telescope without the central obscuration.
HST_RADIUS = (-11.0400, 1.35800)
HST_CONIC = (-1.00230, -1.49686)
HST_SPACING = (-4.90607, 6.40620)
HST_DIAMETER = (2.40000, 0.28112)
HST_EFL = 57.6          # App. D
MAS = math.pi / (180.0 * 3600.0 * 1000.0)


def hst_rc(n_across: int = 64, overlap_factor: float = 1.5, waist_ratio: float = 1.0,
           npix: int = 256, pixel_mas: float = 2.8, wavelength: float = 0.551e-6):
    """The App. B telescope at lambda = 551 nm (App. D), 2.8 mas pixels on its focal plane."""
    msys = MirrorSystem(wavelength, HST_RADIUS, HST_CONIC, HST_SPACING, HST_DIAMETER)
    p = HST_EFL * pixel_mas * MAS
    return msys, Pupil(HST_DIAMETER[0], n_across, overlap_factor, waist_ratio), Detector(npix, npix, p, p)


# The App. B prescription's image distance leaves the real system 108.1 um short of its
# paraxial focus and 110.9 um short of its marginal focus (the RC pair's residual spherical
# aberration).  The telescope sweep puts its detector midway, at the least-RMS-wavefront
# focus, so that its Airy score measures the decomposition rather than that defocus.
HST_REFOCUS = 109.5e-6
# Detector of the telescope sweep: App. D's 2.8 mas pixels, 256^2 (+-7.6 lambda F#).
HST_SWEEP_NPIX = 256


@dataclasses.dataclass(frozen=True)
class MirrorSweep:
    """A batch of GBD instances traced through a mirror sequence (real rays), sharing the
    optics and detector and differing in (N, OF, WR); f_number sets the Airy pattern."""

    system: MirrorSystem
    diameter: float
    f_number: float
    detector: Detector
    n_across: Tuple[int, ...]
    overlap_factor: Tuple[float, ...]
    waist_ratio: Tuple[float, ...]

    @property
    def n_instances(self) -> int:
        return len(self.n_across)

    def pupil(self, k: int) -> Pupil:
        return Pupil(self.diameter, self.n_across[k], self.overlap_factor[k], self.waist_ratio[k])


def telescope_optics(refocus: float = HST_REFOCUS) -> Tuple[MirrorSystem, float, float, Detector]:
    """The App. B telescope at 551 nm with its image plane moved `refocus` metres along the
    axis, its pupil diameter, focal ratio (App. D's focal length) and the sweep's detector."""
    msys, pupil, det = hst_rc(npix=HST_SWEEP_NPIX)
    sp = tuple(HST_SPACING[:-1]) + (HST_SPACING[-1] + refocus,)
    return (dataclasses.replace(msys, spacing=sp), pupil.diameter, HST_EFL / pupil.diameter, det)


def telescope_sweep_from_params(params: Sequence[Tuple[int, float, float]],
                                refocus: float = HST_REFOCUS) -> MirrorSweep:
    msys, D, F, det = telescope_optics(refocus)
    return MirrorSweep(msys, D, F, det, tuple(int(p[0]) for p in params),
                       tuple(float(p[1]) for p in params), tuple(float(p[2]) for p in params))


def telescope_sweep(n_instances: int = 1024, seed: int = SEED_SWEEP) -> MirrorSweep:
    """The seeded 1024-instance draw of the parameter search (same draws as `sweep`) on the
    telescope."""
    sw = sweep(n_instances, seed)
    return telescope_sweep_from_params(list(zip(sw.n_across, sw.overlap_factor, sw.waist_ratio)))


def telescope_grid_sweep() -> MirrorSweep:
    """The reference grid (21 OF x 12 WR x 5 N = 1,260) on the telescope."""
    g = grid_sweep()
    return telescope_sweep_from_params(list(zip(g.n_across, g.overlap_factor, g.waist_ratio)))


def sweep_from_params(params: Sequence[Tuple[int, float, float]]) -> Sweep:
    system, D, det = sweep_optics()
    return Sweep(system, D, det, tuple(int(p[0]) for p in params),
                 tuple(float(p[1]) for p in params), tuple(float(p[2]) for p in params))


def strided_pixels(workload: Workload) -> Tuple[np.ndarray, np.ndarray]:
    """Column / row indices of the oracle's pixel subset (all pixels if no stride)."""
    det = workload.detector
    if workload.oracle_stride is None:
        return np.arange(det.nx), np.arange(det.ny)
    off, step = workload.oracle_stride
    return np.arange(off, det.nx, step), np.arange(off, det.ny, step)


WORKLOADS = {
    "airy_small": airy_small,
    "airy_large": airy_large,
    "tilted_zernike": tilted_zernike,
}


def by_name(name: str) -> Workload:
    return WORKLOADS[name]()


def scaled(workload: Workload, n_across: Optional[int] = None, nx: Optional[int] = None,
           ny: Optional[int] = None, keep_span: bool = True) -> Workload:
    """A smaller copy of a workload (same optics) for oracle-sized parity cases."""
    pupil = workload.pupil
    det = workload.detector
    if n_across is not None:
        pupil = dataclasses.replace(pupil, n_across=n_across)
    if nx is not None or ny is not None:
        nx2 = nx if nx is not None else det.nx
        ny2 = ny if ny is not None else det.ny
        px = det.pitch_x * det.nx / nx2 if keep_span else det.pitch_x
        py = det.pitch_y * det.ny / ny2 if keep_span else det.pitch_y
        det = dataclasses.replace(det, nx=nx2, ny=ny2, pitch_x=px, pitch_y=py)
    return dataclasses.replace(workload, pupil=pupil, detector=det, oracle_stride=None)


def sweep_subset(sw, idx: List[int]):
    """The instances idx of a Sweep or MirrorSweep."""
    return dataclasses.replace(sw, n_across=tuple(sw.n_across[i] for i in idx),
                               overlap_factor=tuple(sw.overlap_factor[i] for i in idx),
                               waist_ratio=tuple(sw.waist_ratio[i] for i in idx))
