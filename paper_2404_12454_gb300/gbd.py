"""Thin ctypes binding of libgbd.so (the C ABI in include/gbd.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
Device buffers are torch tensors (PyTorch provides device memory and streams).  The
binding fails loudly when the compiled library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbd.so")

GBD_OK, GBD_EINVAL, GBD_ECUDA, GBD_ENOMEM, GBD_ETIMEOUT, GBD_EUNSUPPORTED = range(6)
GBD_PREC_F64, GBD_PREC_MIXED = 0, 1
GBD_SCHEME_DIRECT, GBD_SCHEME_ROW_PAIR = 0, 1
GBD_MAX_ZERN = 64
GBD_MAX_MIRRORS = 4
BEAMLET_DOUBLES = 36
TILE = 64

STATUS_NAMES = {0: "GBD_OK", 1: "GBD_EINVAL", 2: "GBD_ECUDA", 3: "GBD_ENOMEM",
                4: "GBD_ETIMEOUT", 5: "GBD_EUNSUPPORTED"}


class GbdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class gbd_system(ctypes.Structure):
    _fields_ = [("wavelength", ctypes.c_double), ("focal_length", ctypes.c_double),
                ("distance", ctypes.c_double), ("zern_radius", ctypes.c_double),
                ("n_zern", ctypes.c_int32), ("noll", ctypes.c_int32 * GBD_MAX_ZERN),
                ("zern_coef", ctypes.c_double * GBD_MAX_ZERN)]


class gbd_pupil(ctypes.Structure):
    _fields_ = [("diameter", ctypes.c_double), ("n_across", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class gbd_mirror_system(ctypes.Structure):
    _fields_ = [("wavelength", ctypes.c_double), ("pupil_offset", ctypes.c_double),
                ("n_mirrors", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("radius", ctypes.c_double * GBD_MAX_MIRRORS),
                ("conic", ctypes.c_double * GBD_MAX_MIRRORS),
                ("spacing", ctypes.c_double * GBD_MAX_MIRRORS)]


class gbd_detector(ctypes.Structure):
    _fields_ = [("pitch_x", ctypes.c_double), ("pitch_y", ctypes.c_double),
                ("rot_x", ctypes.c_double), ("rot_y", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


class gbd_shape(ctypes.Structure):
    _fields_ = [("rows_per_thread", ctypes.c_int32), ("cols_per_thread", ctypes.c_int32),
                ("splits", ctypes.c_int32), ("ms", ctypes.c_float), ("scheme", ctypes.c_int32)]


# Exported symbols of libgbd.so and their ctypes signatures (name -> (restype, argtypes)).
_P = ctypes.c_void_p
_SIGS = {
    "gbd_last_error": (ctypes.c_char_p, []),
    "gbd_version": (ctypes.c_char_p, []),
    "gbd_beamlet_count": (ctypes.c_int32, [ctypes.POINTER(gbd_pupil)]),
    "gbd_sync": (ctypes.c_int, [_P]),
    "gbd_set_wait_limit": (ctypes.c_int, [ctypes.c_uint32]),
    "gbd_trace": (ctypes.c_int, [ctypes.POINTER(gbd_system), ctypes.POINTER(gbd_pupil),
                                 ctypes.c_double, ctypes.c_double, _P, ctypes.c_int32, _P]),
    "gbd_trace_mirrors": (ctypes.c_int, [ctypes.POINTER(gbd_mirror_system),
                                         ctypes.POINTER(gbd_pupil), ctypes.c_double,
                                         ctypes.c_double, _P, ctypes.c_int32, _P]),
    "gbd_field_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.POINTER(gbd_detector),
                                                    ctypes.c_int32]),
    "gbd_field": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(gbd_detector),
                                 ctypes.c_int32, _P, ctypes.c_size_t, _P, _P]),
    "gbd_field_rows_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32,
                                                         ctypes.POINTER(gbd_detector),
                                                         ctypes.c_int32, ctypes.c_int32,
                                                         ctypes.c_int32]),
    "gbd_field_rows": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double,
                                      ctypes.POINTER(gbd_detector), ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _P,
                                      _P]),
    "gbd_truncated_count": (ctypes.c_int32, [ctypes.POINTER(gbd_pupil), ctypes.c_double,
                                             ctypes.c_double, ctypes.POINTER(ctypes.c_int32)]),
    "gbd_trace_truncated": (ctypes.c_int, [ctypes.POINTER(gbd_system), ctypes.POINTER(gbd_pupil),
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, _P,
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P]),
    "gbd_field_truncated_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32,
                                                              ctypes.POINTER(gbd_detector),
                                                              ctypes.c_int32]),
    "gbd_field_truncated": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                           ctypes.POINTER(gbd_detector), ctypes.c_int32, _P,
                                           ctypes.c_size_t, _P, _P]),
    "gbd_project_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "gbd_project": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double,
                                   ctypes.POINTER(gbd_detector), ctypes.c_int32, _P, _P, _P]),
    "gbd_field_set_shape": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(gbd_shape)]),
    "gbd_field_get_shape": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(gbd_detector), ctypes.POINTER(gbd_shape)]),
    "gbd_autotune_field": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double,
                                          ctypes.POINTER(gbd_detector), ctypes.c_int32, _P,
                                          ctypes.c_size_t, _P, _P, ctypes.POINTER(gbd_shape)]),
    "gbd_probe_peaks": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "gbd_sweep_plan_create": (ctypes.c_int, [ctypes.POINTER(gbd_system), ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                             ctypes.POINTER(gbd_detector), ctypes.POINTER(gbd_shape),
                                             ctypes.POINTER(ctypes.c_void_p)]),
    "gbd_sweep_plan_create_mirrors": (ctypes.c_int, [ctypes.POINTER(gbd_mirror_system),
                                                     ctypes.c_double, ctypes.c_double,
                                                     ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.POINTER(ctypes.c_double),
                                                     ctypes.POINTER(ctypes.c_double),
                                                     ctypes.c_int32, ctypes.POINTER(gbd_detector),
                                                     ctypes.POINTER(gbd_shape),
                                                     ctypes.POINTER(ctypes.c_void_p)]),
    "gbd_sweep_workspace_bytes": (ctypes.c_size_t, [_P]),
    "gbd_sweep_set_zones": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
    "gbd_sweep_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "gbd_sweep_bind": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "gbd_sweep_run": (ctypes.c_int, [_P, _P, _P]),
    "gbd_sweep_run_graph": (ctypes.c_int, [_P, _P, _P]),
    "gbd_sweep_autotune": (ctypes.c_int, [ctypes.POINTER(gbd_system), ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                          ctypes.POINTER(gbd_detector), _P, ctypes.c_size_t, _P, _P,
                                          ctypes.POINTER(gbd_shape)]),
    "gbd_sweep_plan_destroy": (None, [_P]),
    "gbd_mlp_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32]),
    "gbd_mlp_pack": (ctypes.c_int, [_P, _P, _P]),
    "gbd_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "gbd_mlp_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, _P]),
    "gbd_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_int32, _P]),
    "gbd_mlp_train": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_size_t, _P]),
    "gbd_mlp_train_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_int32, _P, _P, ctypes.c_size_t, _P]),
    "gbd_field_point_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32,
                                                          ctypes.POINTER(gbd_detector)]),
    "gbd_field_point": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double,
                                       ctypes.POINTER(gbd_detector), _P, ctypes.c_size_t, _P, _P]),
    "gbd_field_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double,
                                         ctypes.POINTER(gbd_detector), ctypes.c_int32, _P, _P]),
    "gbd_timing_enable": (ctypes.c_int, [ctypes.c_int32]),
    "gbd_timing_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "gbd_psf_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(gbd_pupil),
                                                  ctypes.POINTER(gbd_detector), ctypes.c_int32]),
    "gbd_psf": (ctypes.c_int, [ctypes.POINTER(gbd_system), ctypes.POINTER(gbd_pupil),
                               ctypes.c_double, ctypes.c_double, ctypes.POINTER(gbd_detector),
                               ctypes.c_int32, _P, ctypes.c_size_t, _P, _P]),
}

_lib = None


def lib():
    """The loaded libgbd.so.  Raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != GBD_OK:
        raise GbdError(status, lib().gbd_last_error().decode())


def _stream(stream=None):
    """cudaStream_t of a torch stream, an integer handle, or torch's current stream."""
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


# ---------------------------------------------------------------- structures --

def make_system(system) -> gbd_system:
    """gbd_system from an object with wavelength, focal_length, distance, noll, ..."""
    s = gbd_system()
    s.wavelength = system.wavelength
    s.focal_length = system.focal_length
    s.distance = system.distance
    noll = list(getattr(system, "noll", ()))
    coef = list(getattr(system, "zern_coef", ()))
    if len(noll) > GBD_MAX_ZERN:
        raise ValueError("too many Zernike terms")
    s.n_zern = len(noll)
    s.zern_radius = getattr(system, "zern_radius", 1.0) if noll else 1.0
    for t, (j, c) in enumerate(zip(noll, coef)):
        s.noll[t] = int(j)
        s.zern_coef[t] = float(c)
    return s


def make_mirror_system(msys) -> gbd_mirror_system:
    """gbd_mirror_system from an object with wavelength, pupil_offset, radius, conic, spacing."""
    n = len(msys.radius)
    if not (len(msys.conic) == n and len(msys.spacing) == n):
        raise ValueError("radius, conic and spacing must have one entry per mirror")
    if n > GBD_MAX_MIRRORS:
        raise ValueError("too many mirrors")
    s = gbd_mirror_system()
    s.wavelength = msys.wavelength
    s.pupil_offset = msys.pupil_offset
    s.n_mirrors = n
    for k in range(n):
        s.radius[k] = float(msys.radius[k])
        s.conic[k] = float(msys.conic[k])
        s.spacing[k] = float(msys.spacing[k])
    return s


def make_pupil(pupil) -> gbd_pupil:
    return gbd_pupil(float(pupil.diameter), int(pupil.n_across), 0)


def make_detector(det) -> gbd_detector:
    return gbd_detector(float(det.pitch_x), float(det.pitch_y), float(det.rot_x), float(det.rot_y),
                        int(det.nx), int(det.ny))


# ------------------------------------------------------------ C ABI mirrors --

def gbd_version() -> str:
    return lib().gbd_version().decode()


def gbd_beamlet_count(pupil) -> int:
    return int(lib().gbd_beamlet_count(ctypes.byref(make_pupil(pupil))))


def gbd_sync(stream=None) -> None:
    _check(lib().gbd_sync(_stream(stream)))


def gbd_set_wait_limit(spins: int) -> None:
    _check(lib().gbd_set_wait_limit(int(spins)))


def gbd_trace(system, pupil, overlap_factor: float, waist_ratio: float, out, stream=None) -> int:
    """Traces the pupil into ``out`` (float64 CUDA tensor [capacity, 36]); returns n."""
    n = gbd_beamlet_count(pupil)
    cap = out.shape[0] if out is not None else 0
    _check(lib().gbd_trace(ctypes.byref(make_system(system)), ctypes.byref(make_pupil(pupil)),
                           float(overlap_factor), float(waist_ratio), _ptr(out), int(cap),
                           _stream(stream)))
    return n


def gbd_trace_mirrors(msys, pupil, overlap_factor: float, waist_ratio: float, out,
                      stream=None) -> int:
    """Traces the pupil through conic mirrors into ``out`` (float64 [capacity, 36])."""
    n = gbd_beamlet_count(pupil)
    cap = out.shape[0] if out is not None else 0
    _check(lib().gbd_trace_mirrors(ctypes.byref(make_mirror_system(msys)),
                                   ctypes.byref(make_pupil(pupil)), float(overlap_factor),
                                   float(waist_ratio), _ptr(out), int(cap), _stream(stream)))
    return n


def gbd_field_workspace_bytes(n_beamlets: int, detector, precision: int) -> int:
    return int(lib().gbd_field_workspace_bytes(int(n_beamlets),
                                               ctypes.byref(make_detector(detector)),
                                               int(precision)))


def gbd_field(beamlets, n_beamlets: int, wavelength: float, detector, precision: int,
              workspace, field_out, stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbd_field(_ptr(beamlets), int(n_beamlets), float(wavelength),
                           ctypes.byref(make_detector(detector)), int(precision),
                           _ptr(workspace), ctypes.c_size_t(ws_bytes), _ptr(field_out),
                           _stream(stream)))


def gbd_field_rows_workspace_bytes(n_beamlets: int, detector, row_begin: int, row_end: int,
                                   precision: int) -> int:
    return int(lib().gbd_field_rows_workspace_bytes(int(n_beamlets),
                                                    ctypes.byref(make_detector(detector)),
                                                    int(row_begin), int(row_end),
                                                    int(precision)))


def gbd_field_rows(beamlets, n_beamlets: int, wavelength: float, detector, row_begin: int,
                   row_end: int, precision: int, workspace, field_out, stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbd_field_rows(_ptr(beamlets), int(n_beamlets), float(wavelength),
                                ctypes.byref(make_detector(detector)), int(row_begin),
                                int(row_end), int(precision), _ptr(workspace),
                                ctypes.c_size_t(ws_bytes), _ptr(field_out), _stream(stream)))


def gbd_truncated_count(pupil, overlap_factor: float, margin: float = 3.0) -> Tuple[int, int]:
    """(beamlets, edge beamlets) of the truncated decomposition; (-1, 0) for bad input."""
    ne = ctypes.c_int32(0)
    n = int(lib().gbd_truncated_count(ctypes.byref(make_pupil(pupil)), float(overlap_factor),
                                      float(margin), ctypes.byref(ne)))
    return n, int(ne.value)


def gbd_trace_truncated(system, pupil, overlap_factor: float, waist_ratio: float, margin: float,
                        out, stream=None) -> int:
    """Fills `out` (float64 CUDA tensor [>= n, 36]); returns the edge count."""
    ne = ctypes.c_int32(0)
    _check(lib().gbd_trace_truncated(ctypes.byref(make_system(system)), ctypes.byref(make_pupil(pupil)),
                                     float(overlap_factor), float(waist_ratio), float(margin),
                                     _ptr(out), int(out.shape[0]), ctypes.byref(ne), _stream(stream)))
    return int(ne.value)


def gbd_field_truncated_workspace_bytes(n_beamlets: int, n_edge: int, detector,
                                        precision: int) -> int:
    return int(lib().gbd_field_truncated_workspace_bytes(int(n_beamlets), int(n_edge),
                                                         ctypes.byref(make_detector(detector)),
                                                         int(precision)))


def gbd_field_truncated(beamlets, n_beamlets: int, n_edge: int, wavelength: float, detector,
                        precision: int, workspace, field_out, stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbd_field_truncated(_ptr(beamlets), int(n_beamlets), int(n_edge),
                                     float(wavelength), ctypes.byref(make_detector(detector)),
                                     int(precision), _ptr(workspace), ctypes.c_size_t(ws_bytes),
                                     _ptr(field_out), _stream(stream)))


def gbd_project_bytes(n_beamlets: int, precision: int) -> int:
    return int(lib().gbd_project_bytes(int(n_beamlets), int(precision)))


def gbd_project(beamlets, n_beamlets: int, wavelength: float, detector, precision: int, coeffs,
                wide_flag=None, stream=None) -> None:
    """Projected records into ``coeffs``; ``wide_flag`` (int32 CUDA tensor, zeroed) gets
    the projection's flag bits (mixed only): 0 some beamlet's phase can exceed 128 rad on
    the detector, 1 the row-pair scheme must fall back to direct evaluation, 2 the
    amplitude may not be carried along a row, 3 the field has a uv term, 4 the row triples
    and quadruples must hand the field to the row pairs."""
    _check(lib().gbd_project(_ptr(beamlets), int(n_beamlets), float(wavelength),
                             ctypes.byref(make_detector(detector)), int(precision), _ptr(coeffs),
                             _ptr(wide_flag), _stream(stream)))


def gbd_field_set_shape(precision: int, rows: int, cols: int, splits: int = 0,
                        scheme: int = GBD_SCHEME_DIRECT) -> None:
    sh = gbd_shape(int(rows), int(cols), int(splits), 0.0, int(scheme))
    _check(lib().gbd_field_set_shape(int(precision), ctypes.byref(sh)))


def gbd_field_reset_shape(precision: int) -> None:
    _check(lib().gbd_field_set_shape(int(precision), None))


def gbd_field_get_shape(precision: int, n_beamlets: int, detector) -> Tuple[int, int, int, int]:
    sh = gbd_shape()
    _check(lib().gbd_field_get_shape(int(precision), int(n_beamlets),
                                     ctypes.byref(make_detector(detector)), ctypes.byref(sh)))
    return sh.rows_per_thread, sh.cols_per_thread, sh.splits, sh.scheme


def gbd_autotune_field(beamlets, n_beamlets: int, wavelength: float, detector, precision: int,
                       workspace, field_out, stream=None) -> Tuple[int, int, int, float, int]:
    sh = gbd_shape()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().gbd_autotune_field(_ptr(beamlets), int(n_beamlets), float(wavelength),
                                    ctypes.byref(make_detector(detector)), int(precision),
                                    _ptr(workspace), ctypes.c_size_t(ws_bytes), _ptr(field_out),
                                    _stream(stream), ctypes.byref(sh)))
    return sh.rows_per_thread, sh.cols_per_thread, sh.splits, float(sh.ms), sh.scheme


def gbd_probe_peaks() -> dict:
    out = (ctypes.c_double * 5)()
    _check(lib().gbd_probe_peaks(out))
    return dict(zip(("ex2", "sin", "cos", "ffma", "dfma"), list(out)))


NOALLOC_SCRATCH_BYTES = 32 << 20


def gbd_field_noalloc(beamlets, n_beamlets: int, wavelength: float, detector, precision: int,
                      field_out, stream=None) -> None:
    """gbd_field without a workspace: scratch is a fixed 32 MiB array inside the library,
    for callers that may not allocate device memory.  Calls share that array, so calls
    that overlap on the GPU must be serialised; the first call on a device should come
    before any stream capture."""
    _check(lib().gbd_field_noalloc(_ptr(beamlets), int(n_beamlets), float(wavelength),
                                   ctypes.byref(make_detector(detector)), int(precision),
                                   _ptr(field_out), _stream(stream)))


def _instance_arrays(n_across, overlap_factor, waist_ratio):
    n = len(n_across)
    if not (len(overlap_factor) == n and len(waist_ratio) == n):
        raise ValueError("instance arrays differ in length")
    a = (ctypes.c_int32 * n)(*[int(v) for v in n_across])
    b = (ctypes.c_double * n)(*[float(v) for v in overlap_factor])
    c = (ctypes.c_double * n)(*[float(v) for v in waist_ratio])
    return n, a, b, c


class SweepPlan:
    """A bound batched sweep (gbd_sweep_plan_* / gbd_sweep_bind): n instances sharing
    the optics and detector, each with its own (n_across, overlap_factor, waist_ratio);
    run() returns the Airy scores as a float64 CUDA tensor."""

    def __init__(self, system, diameter, n_across, overlap_factor, waist_ratio, detector,
                 shape: Optional[Tuple[int, ...]] = None, stream=None, device="cuda",
                 zones: Optional[Sequence[Tuple[float, float]]] = None,
                 f_number: Optional[float] = None):
        """shape: (rows, cols[, scheme]) per thread; None = the library's sweep default (row
        triples on 8 columns or row pairs on 4, fitted to the detector's width).  A mirror
        system (workloads.MirrorSystem) traces every instance by real rays through it
        (gbd_sweep_plan_create_mirrors) and needs the system's f_number."""
        import torch
        n, a, b, c = _instance_arrays(n_across, overlap_factor, waist_ratio)
        self.n = n
        self._plan = ctypes.c_void_p()
        sh = (gbd_shape(shape[0], shape[1], 1, 0.0, shape[2] if len(shape) > 2 else 0)
              if shape else None)
        if hasattr(system, "radius"):
            if f_number is None:
                raise ValueError("a mirror sweep needs the system's f_number")
            _check(lib().gbd_sweep_plan_create_mirrors(
                ctypes.byref(make_mirror_system(system)), float(diameter), float(f_number), a, b,
                c, n, ctypes.byref(make_detector(detector)), ctypes.byref(sh) if sh else None,
                ctypes.byref(self._plan)))
        else:
            _check(lib().gbd_sweep_plan_create(ctypes.byref(make_system(system)), float(diameter),
                                               a, b, c, n, ctypes.byref(make_detector(detector)),
                                               ctypes.byref(sh) if sh else None,
                                               ctypes.byref(self._plan)))
        self.n_regions = 1
        if zones:
            lo = (ctypes.c_double * len(zones))(*[float(z[0]) for z in zones])
            hi = (ctypes.c_double * len(zones))(*[float(z[1]) for z in zones])
            _check(lib().gbd_sweep_set_zones(self._plan, len(zones), lo, hi))
            self.n_regions = 1 + len(zones)
        self.bytes = int(lib().gbd_sweep_workspace_bytes(self._plan))
        self.ws = torch.empty(self.bytes, dtype=torch.uint8, device=device)
        self.scores = torch.empty(n * self.n_regions, dtype=torch.float64, device=device)
        _check(lib().gbd_sweep_bind(self._plan, _ptr(self.ws), ctypes.c_size_t(self.bytes),
                                    _stream(stream)))
        ev, nb, items = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().gbd_sweep_info(self._plan, ctypes.byref(ev), ctypes.byref(nb),
                                    ctypes.byref(items)))
        self.evals, self.beamlets, self.items = float(ev.value), int(nb.value), int(items.value)

    def run(self, stream=None, graph: bool = False):
        """Scores as a float64 CUDA tensor: [n] without zones, [n, 1 + zones] with."""
        fn = lib().gbd_sweep_run_graph if graph else lib().gbd_sweep_run
        _check(fn(self._plan, _ptr(self.scores), _stream(stream)))
        return self.scores if self.n_regions == 1 else self.scores.view(self.n, self.n_regions)

    def close(self):
        if getattr(self, "_plan", None) is not None and self._plan.value:
            lib().gbd_sweep_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_plan(sw, shape=None, stream=None, zones=None) -> SweepPlan:
    """SweepPlan for a workloads.Sweep or workloads.MirrorSweep description."""
    return SweepPlan(sw.system, sw.diameter, sw.n_across, sw.overlap_factor, sw.waist_ratio,
                     sw.detector, shape, stream, zones=zones,
                     f_number=getattr(sw, "f_number", None))


def gbd_sweep_autotune(system, diameter, n_across, overlap_factor, waist_ratio, detector,
                       workspace, scores, stream=None) -> Tuple[int, int, float, int]:
    n, a, b, c = _instance_arrays(n_across, overlap_factor, waist_ratio)
    sh = gbd_shape()
    _check(lib().gbd_sweep_autotune(ctypes.byref(make_system(system)), float(diameter), a, b, c, n,
                                    ctypes.byref(make_detector(detector)), _ptr(workspace),
                                    ctypes.c_size_t(workspace.numel()), _ptr(scores),
                                    _stream(stream), ctypes.byref(sh)))
    return sh.rows_per_thread, sh.cols_per_thread, float(sh.ms), sh.scheme


def gbd_field_point_workspace_bytes(n_beamlets: int, detector) -> int:
    return int(lib().gbd_field_point_workspace_bytes(int(n_beamlets),
                                                     ctypes.byref(make_detector(detector))))


def gbd_field_point(beamlets, n_beamlets: int, wavelength: float, detector, workspace, field_out,
                    stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().gbd_field_point(_ptr(beamlets), int(n_beamlets), float(wavelength),
                                 ctypes.byref(make_detector(detector)), _ptr(workspace),
                                 ctypes.c_size_t(ws_bytes), _ptr(field_out), _stream(stream)))


def field_point(beamlets, wavelength: float, detector, stream=None):
    """Point-evaluation field (complex128 CUDA tensor [ny, nx])."""
    import torch
    n = int(beamlets.shape[0])
    out = torch.empty((detector.ny, detector.nx), dtype=torch.complex128, device=beamlets.device)
    ws = torch.empty(max(256, gbd_field_point_workspace_bytes(n, detector)), dtype=torch.uint8,
                     device=beamlets.device)
    gbd_field_point(beamlets, n, wavelength, detector, ws, out, stream)
    return out


MLP_PARAMS = 50177


def gbd_mlp_workspace_bytes(batch: int) -> int:
    return int(lib().gbd_mlp_workspace_bytes(int(batch)))


def gbd_mlp_pack(master, weights, stream=None) -> None:
    _check(lib().gbd_mlp_pack(_ptr(master), _ptr(weights), _stream(stream)))


def gbd_mlp_forward(weights, x, y, stream=None) -> None:
    _check(lib().gbd_mlp_forward(_ptr(weights), _ptr(x), int(x.shape[0]), _ptr(y), _stream(stream)))


def gbd_mlp_grad(weights, x, target, grad, loss, workspace, stream=None) -> None:
    _check(lib().gbd_mlp_grad(_ptr(weights), _ptr(x), _ptr(target), int(x.shape[0]), _ptr(grad),
                              _ptr(loss), _ptr(workspace), ctypes.c_size_t(workspace.numel()),
                              _stream(stream)))


def gbd_mlp_adam(master, weights, m, v, grad, lr, beta1, beta2, eps, step, stream=None) -> None:
    _check(lib().gbd_mlp_adam(_ptr(master), _ptr(weights), _ptr(m), _ptr(v), _ptr(grad),
                              float(lr), float(beta1), float(beta2), float(eps), int(step),
                              _stream(stream)))


def gbd_mlp_train(master, weights, m, v, x, target, lr, beta1, beta2, eps, first_step, steps,
                  loss, workspace, stream=None) -> None:
    _check(lib().gbd_mlp_train(_ptr(master), _ptr(weights), _ptr(m), _ptr(v), _ptr(x),
                               _ptr(target), int(x.shape[0]), float(lr), float(beta1),
                               float(beta2), float(eps), int(first_step), int(steps), _ptr(loss),
                               _ptr(workspace), ctypes.c_size_t(workspace.numel()),
                               _stream(stream)))


def gbd_mlp_train_step(master, weights, m, v, x, target, lr, beta1, beta2, eps, step, loss,
                       workspace, stream=None) -> None:
    _check(lib().gbd_mlp_train_step(_ptr(master), _ptr(weights), _ptr(m), _ptr(v), _ptr(x),
                                    _ptr(target), int(x.shape[0]), float(lr), float(beta1),
                                    float(beta2), float(eps), int(step), _ptr(loss),
                                    _ptr(workspace), ctypes.c_size_t(workspace.numel()),
                                    _stream(stream)))


TIMING_KINDS = ("field_mixed", "field_f64", "project", "reduce", "point", "trace")


def gbd_timing_enable(on: bool) -> None:
    _check(lib().gbd_timing_enable(1 if on else 0))


def gbd_timing_read() -> dict:
    ms = (ctypes.c_double * len(TIMING_KINDS))()
    n = (ctypes.c_int64 * len(TIMING_KINDS))()
    _check(lib().gbd_timing_read(ms, n))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(TIMING_KINDS)}


def gbd_psf_workspace_bytes(pupil, detector, precision: int) -> int:
    return int(lib().gbd_psf_workspace_bytes(ctypes.byref(make_pupil(pupil)),
                                             ctypes.byref(make_detector(detector)), int(precision)))


def gbd_psf(system, pupil, overlap_factor: float, waist_ratio: float, detector, precision: int,
            workspace, host_out, stream=None) -> None:
    """Trace + field + copy into ``host_out`` (a CPU tensor, pinned for async copies)."""
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib().gbd_psf(ctypes.byref(make_system(system)), ctypes.byref(make_pupil(pupil)),
                         float(overlap_factor), float(waist_ratio),
                         ctypes.byref(make_detector(detector)), int(precision), _ptr(workspace),
                         ctypes.c_size_t(ws_bytes), _ptr(host_out), _stream(stream)))


# ------------------------------------------------------------ conveniences --

def trace(system, pupil, device="cuda", stream=None):
    """Beamlet table as a float64 CUDA tensor [n, 36] (gbd_trace)."""
    import torch
    n = gbd_beamlet_count(pupil)
    out = torch.empty((max(n, 1), BEAMLET_DOUBLES), dtype=torch.float64, device=device)
    gbd_trace(system, pupil, pupil.overlap_factor, pupil.waist_ratio, out, stream)
    return out[:n]


def trace_mirrors(msys, pupil, device="cuda", stream=None):
    """Beamlet table of a pupil in front of conic mirrors (gbd_trace_mirrors)."""
    import torch
    n = gbd_beamlet_count(pupil)
    out = torch.empty((max(n, 1), BEAMLET_DOUBLES), dtype=torch.float64, device=device)
    gbd_trace_mirrors(msys, pupil, pupil.overlap_factor, pupil.waist_ratio, out, stream)
    return out[:n]


def workspace(n_beamlets: int, detector, precision: int, device="cuda"):
    import torch
    nbytes = gbd_field_workspace_bytes(n_beamlets, detector, precision)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def field(beamlets, wavelength: float, detector, precision: int = GBD_PREC_MIXED, ws=None,
          out=None, stream=None):
    """Complex field [ny, nx] (complex64 mixed / complex128 FP64) as a CUDA tensor."""
    import torch
    n = int(beamlets.shape[0])
    dtype = torch.complex64 if precision == GBD_PREC_MIXED else torch.complex128
    if out is None:
        out = torch.empty((detector.ny, detector.nx), dtype=dtype, device=beamlets.device)
    if ws is None:
        ws = workspace(n, detector, precision, beamlets.device)
    gbd_field(beamlets, n, wavelength, detector, precision, ws, out, stream)
    return out


def field_rows(beamlets, wavelength: float, detector, row_begin: int, row_end: int,
               precision: int = GBD_PREC_MIXED, ws=None, out=None, stream=None):
    """Detector rows [row_begin, row_end) of the field, [row_end - row_begin, nx], as a
    CUDA tensor: the same bits as those rows of ``field``."""
    import torch
    n = int(beamlets.shape[0])
    dtype = torch.complex64 if precision == GBD_PREC_MIXED else torch.complex128
    if out is None:
        out = torch.empty((row_end - row_begin, detector.nx), dtype=dtype, device=beamlets.device)
    if ws is None:
        nbytes = gbd_field_rows_workspace_bytes(n, detector, row_begin, row_end, precision)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=beamlets.device)
    gbd_field_rows(beamlets, n, wavelength, detector, row_begin, row_end, precision, ws, out,
                   stream)
    return out


def trace_truncated(system, pupil, margin: float = 3.0, device="cuda", stream=None):
    """(beamlet table of the truncated decomposition, edge count): whole beamlets first."""
    import torch
    n, _ = gbd_truncated_count(pupil, pupil.overlap_factor, margin)
    out = torch.empty((max(n, 1), BEAMLET_DOUBLES), dtype=torch.float64, device=device)
    ne = gbd_trace_truncated(system, pupil, pupil.overlap_factor, pupil.waist_ratio, margin, out,
                             stream)
    return out[:n], ne


def field_truncated(beamlets, n_edge: int, wavelength: float, detector,
                    precision: int = GBD_PREC_MIXED, stream=None):
    """Field [ny, nx] of a truncated decomposition (untilted detector) as a CUDA tensor."""
    import torch
    n = int(beamlets.shape[0])
    dtype = torch.complex64 if precision == GBD_PREC_MIXED else torch.complex128
    out = torch.empty((detector.ny, detector.nx), dtype=dtype, device=beamlets.device)
    nbytes = gbd_field_truncated_workspace_bytes(n, n_edge, detector, precision)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=beamlets.device)
    gbd_field_truncated(beamlets, n, n_edge, wavelength, detector, precision, ws, out, stream)
    return out


def psf(system, pupil, detector, precision: int = GBD_PREC_MIXED, stream=None):
    """Trace + field in one call; returns the complex field as a CUDA tensor."""
    b = trace(system, pupil, stream=stream)
    return field(b, system.wavelength, detector, precision, stream=stream)


def unpack(rec: np.ndarray) -> dict:
    """Named views of one gbd_beamlet record (36 doubles)."""
    r = np.asarray(rec, dtype=np.float64)
    return dict(rho=r[0:2], theta=r[2:4], path=r[4], amp=complex(r[5], r[6]),
                P=(r[7:15:2] + 1j * r[8:15:2]).reshape(2, 2), A=r[15:19].reshape(2, 2),
                B=r[19:23].reshape(2, 2), C=r[23:27].reshape(2, 2), D=r[27:31].reshape(2, 2),
                center=r[31:33], weight=r[33], waist=r[34], edge_distance=r[35])
