"""CUDA path (through the C ABI) against the FP64 CPU oracle.

Trace records field by field; fields by relative L2 over all compared pixels:
<= 1e-11 for the FP64 path, <= 2e-5 for the mixed path (FP32 per-pixel phase and MUFU
ex2/sin/cos, compensated sum).  Sizes span several beamlet tiles and pixel blocks with
ragged tails; the two workloads at full size are compared on pixel subsets the oracle
computes one by one.
"""
import math

import numpy as np
import pytest

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
    yield
    gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)
    gbd.gbd_field_reset_shape(gbd.GBD_PREC_F64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_trace(wl):
    b = gbd.trace(wl.system, wl.pupil)
    gbd.gbd_sync()
    return b


def gpu_field(b, wl, prec):
    E = gbd.field(b, wl.system.wavelength, wl.detector, prec)
    gbd.gbd_sync()
    return E.cpu().numpy().astype(np.complex128)


def small_cases():
    airy = W.airy_small()
    tz = W.tilted_zernike()
    return {
        "airy_small": airy,
        "airy_ragged": W.scaled(airy, n_across=23, nx=97, ny=45),
        "tilted_zernike_small": W.scaled(tz, n_across=24, nx=80, ny=72),
        "defocused": W.Workload("defocused", W.System(1e-6, 0.024, 0.0246), W.Pupil(2.4e-3, 16, 1.2, 2.0),
                                W.Detector(70, 66, 1.5e-6, 1.2e-6)),
        "tilted_defocused": W.Workload("tilted_defocused", W.System(0.633e-6, 0.012, 0.0121),
                                       W.Pupil(2.4e-3, 20, 2.0, 1.2),
                                       W.Detector(64, 50, 0.4e-6, 0.5e-6, math.radians(-12),
                                                  math.radians(7))),
    }


@pytest.mark.parametrize("name", list(small_cases()))
def test_trace_records_match_oracle(name):
    wl = small_cases()[name]
    g = gpu_trace(wl).cpu().numpy()
    o = oracle.trace(wl.system, wl.pupil)
    assert g.shape[0] == o.shape[0]
    for rg, ro in zip(g, o):
        a, b = gbd.unpack(rg), oracle.unpack(ro)
        assert np.allclose(a["center"], b["r"], rtol=0, atol=1e-18)
        assert abs(a["weight"] - b["a"]) <= 1e-15 * b["a"]
        assert abs(a["waist"] - b["w0"]) <= 1e-18
        assert np.allclose(a["rho"], b["rho"], rtol=0, atol=1e-16)
        assert np.allclose(a["theta"], b["theta"], rtol=0, atol=1e-14)
        assert abs(a["path"] - b["L"]) <= 1e-17
        for k in "ABCD":
            scale = max(1.0, np.abs(b[k]).max())
            assert np.allclose(a[k], b[k], rtol=0, atol=1e-10 * scale), k
        assert np.allclose(a["P"], b["P"], rtol=0, atol=1e-10 * np.abs(b["P"]).max())
        assert abs(a["amp"] - b["alpha"]) <= 1e-12 * abs(b["alpha"])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(small_cases()))
def test_field_matches_oracle(name, prec):
    wl = small_cases()[name]
    b = gpu_trace(wl)
    E = gpu_field(b, wl, prec)
    o = oracle.trace(wl.system, wl.pupil)
    Eo = oracle.field(o, wl.system, wl.detector)
    err = rel_l2(E, Eo)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_airy_large_sampled(prec):
    """512 x 512 pixels, 51,468 beamlets on the GPU; oracle on a strided 32 x 32 sample."""
    wl = W.airy_large()
    b = gpu_trace(wl)
    E = gpu_field(b, wl, prec)
    cols = np.arange(3, 512, 16)
    rows = np.arange(5, 512, 16)
    o = oracle.trace(wl.system, wl.pupil)
    Eo = oracle.field(o, wl.system, wl.detector, cols, rows)
    err = rel_l2(E[np.ix_(rows, cols)], Eo)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("name", ["airy_large", "tilted_zernike"])
def test_full_size_in_the_autotuned_launch_configuration(name):
    """The configuration bench.py times: the autotuner's pick (shape, splits, scheme) on
    the full-size workload, checked on the oracle's strided pixel sample."""
    import torch
    wl = W.by_name(name)
    b = gpu_trace(wl)
    prec = gbd.GBD_PREC_MIXED
    ws = torch.empty(640 << 20, dtype=torch.uint8, device="cuda")
    out = torch.empty((wl.detector.ny, wl.detector.nx), dtype=torch.complex64, device="cuda")
    try:
        gbd.gbd_autotune_field(b, b.shape[0], wl.system.wavelength, wl.detector, prec, ws, out)
        del ws
        E = gpu_field(b, wl, prec)
    finally:
        gbd.gbd_field_reset_shape(prec)
    if name == "airy_large":
        cols, rows = np.arange(3, 512, 16), np.arange(5, 512, 16)
    else:
        cols, rows = W.strided_pixels(wl)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector, cols, rows)
    assert rel_l2(E[np.ix_(rows, cols)], Eo) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_tilted_zernike_subset(prec):
    """1024 x 1024 tilted, aberrated detector; oracle on the 64 x 64 strided subset."""
    wl = W.tilted_zernike()
    b = gpu_trace(wl)
    E = gpu_field(b, wl, prec)
    cols, rows = W.strided_pixels(wl)
    o = oracle.trace(wl.system, wl.pupil)
    Eo = oracle.field(o, wl.system, wl.detector, cols, rows)
    err = rel_l2(E[np.ix_(rows, cols)], Eo)
    assert err <= TOL[prec], err


# ----------------------------------------------------------------- edge cases --

@pytest.mark.parametrize("prec", PRECS)
def test_zero_beamlets_gives_zero_field(prec):
    import torch
    det = W.Detector(37, 11, 1e-6, 1e-6)
    dtype = torch.complex64 if prec == gbd.GBD_PREC_MIXED else torch.complex128
    out = torch.full((11, 37), 7.0, dtype=dtype, device="cuda")
    empty = torch.empty((0, 36), dtype=torch.float64, device="cuda")
    gbd.gbd_field(empty, 0, 1e-6, det, prec, None, out)
    gbd.gbd_sync()
    assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 300), (300, 1), (33, 7)])
def test_degenerate_detectors(prec, shape):
    nx, ny = shape
    wl = W.Workload("edge", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 9, 1.5, 1.5),
                    W.Detector(nx, ny, 0.9e-6, 1.1e-6))
    b = gpu_trace(wl)
    E = gpu_field(b, wl, prec)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    assert rel_l2(E, Eo) <= TOL[prec]


@pytest.mark.parametrize("rows,cols", [(4, 8), (2, 16), (8, 4)])
@pytest.mark.parametrize("shape", [(1, 1), (1, 300), (300, 1), (33, 7), (128, 96), (300, 40)])
def test_fp64_shared_row_recurrence(shape, rows, cols):
    """The FP64 row segments whose row factors come from a warp table (beamlets without a
    uv term: the untilted thin-lens system) on one-row, one-column (narrow: the per-row
    fallback), ragged and wide detectors, against the oracle at the FP64 tolerance."""
    nx, ny = shape
    wl = W.Workload("edge", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 9, 1.5, 1.5),
                    W.Detector(nx, ny, 0.9e-6, 1.1e-6))
    b = gpu_trace(wl)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    try:
        for splits in (1, 3):
            gbd.gbd_field_set_shape(gbd.GBD_PREC_F64, rows, cols, splits, gbd.GBD_SCHEME_DIRECT)
            E = gpu_field(b, wl, gbd.GBD_PREC_F64)
            assert rel_l2(E, Eo) <= TOL[gbd.GBD_PREC_F64], (rows, cols, splits)
    finally:
        gbd.gbd_field_reset_shape(gbd.GBD_PREC_F64)


@pytest.mark.parametrize("rows,cols", [(3, 8), (4, 4)])
@pytest.mark.parametrize("shape", [(1, 1), (1, 300), (300, 1), (33, 7)])
def test_degenerate_detectors_with_row_triples_and_quadruples(shape, rows, cols):
    """The multi-row kernels on detectors of one row or column and on a ragged 33 x 7
    detector (every thread's later rows or columns off the detector)."""
    nx, ny = shape
    wl = W.Workload("edge", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 9, 1.5, 1.5),
                    W.Detector(nx, ny, 0.9e-6, 1.1e-6))
    b = gpu_trace(wl)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    try:
        gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, rows, cols, 1, gbd.GBD_SCHEME_ROW_PAIR)
        E = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
    finally:
        gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)
    assert rel_l2(E, Eo) <= TOL[gbd.GBD_PREC_MIXED]


@pytest.mark.parametrize("prec", PRECS)
def test_single_beamlet_free_space(prec):
    """One beamlet, no lens: the textbook Gaussian through the whole CUDA path."""
    lam, D = 1e-6, 1e-3
    zR = math.pi * (D / 2) ** 2 / lam
    wl = W.Workload("one", W.System(lam, math.inf, 3 * zR), W.Pupil(D, 1, 1.0, 1.0),
                    W.Detector(40, 40, 0.2e-3, 0.2e-3))
    b = gpu_trace(wl)
    E = gpu_field(b, wl, prec)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    assert rel_l2(E, Eo) <= TOL[prec]


def test_mixed_is_deterministic():
    wl = W.airy_small()
    b = gpu_trace(wl)
    E1 = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
    E2 = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
    assert np.array_equal(E1, E2)


@pytest.mark.parametrize("prec", PRECS)
def test_every_shape_and_split_matches(prec):
    """Each compiled launch shape and several beamlet splits give the oracle's field."""
    wl = small_cases()["tilted_zernike_small"]
    b = gpu_trace(wl)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    D, P = gbd.GBD_SCHEME_DIRECT, gbd.GBD_SCHEME_ROW_PAIR
    shapes = ([(1, 4, D), (2, 2, D), (2, 4, D), (4, 2, D), (2, 2, P), (2, 4, P), (2, 8, P),
               (3, 8, P), (4, 8, P), (4, 4, P)]
              if prec == gbd.GBD_PREC_MIXED
              else [(1, 2, D), (2, 2, D), (1, 8, D), (2, 8, D), (1, 16, D), (1, 32, D),
                    (4, 8, D), (2, 16, D), (8, 4, D)])
    try:
        for rows, cols, scheme in shapes:
            for splits in (1, 2, 5):
                gbd.gbd_field_set_shape(prec, rows, cols, splits, scheme)
                E = gpu_field(b, wl, prec)
                assert rel_l2(E, Eo) <= TOL[prec], (rows, cols, splits, scheme)
    finally:
        gbd.gbd_field_reset_shape(prec)


def projection_flags(b, wl):
    import torch
    n = b.shape[0]
    coef = torch.empty(gbd.gbd_project_bytes(n, gbd.GBD_PREC_MIXED), dtype=torch.uint8,
                       device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    gbd.gbd_project(b, n, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED, coef, flag)
    gbd.gbd_sync()
    return int(flag.item())


@pytest.mark.parametrize("name", list(small_cases()) + ["airy_large", "tilted_zernike"])
def test_row_pair_scheme_is_not_flagged_on_the_workloads(name):
    """The row-pair recurrence applies to every workload (no fallback to direct); on the
    full-size workloads the amplitude recurrence along rows applies too (the narrow-phase
    instantiation runs)."""
    wl = small_cases()[name] if name in small_cases() else W.by_name(name)
    f = projection_flags(gpu_trace(wl), wl)
    assert f & 2 == 0
    if name in ("airy_large", "tilted_zernike"):
        assert f & 7 == 0
    # the untilted thin lens has no uv term (every column factor T is exactly 1, so the
    # instantiation without its update runs); the tilted, aberrated system has one
    if name in ("airy_small", "airy_large"):
        assert f & 8 == 0
    if name == "tilted_zernike":
        assert f & 8


def near_wide_case():
    """Beamlets about 41 lambda F# wide (64 across, OF 1.0) on a 616^2 detector at the
    large Airy workload's pitch (+-24 lambda F#): their phases reach ~123 rad on the
    detector where their amplitude is still large, just under the 128 rad bound above
    which the projection asks for exact per-pixel range reduction."""
    big = W.airy_large()
    p = big.detector.pitch_x
    return W.Workload("near_wide", big.system, W.Pupil(2.4e-3, 64, 1.0, 1.0),
                      W.Detector(616, 616, p, p))


@pytest.mark.parametrize("shape", [None, (2, 4, gbd.GBD_SCHEME_DIRECT),
                                   (2, 8, gbd.GBD_SCHEME_ROW_PAIR)])
def test_phases_just_under_the_wide_bound(shape):
    """The narrow kernels take sin/cos of unreduced phases up to the bound (the MUFU error
    grows with the argument).  On the case above the projection does not flag the field
    as wide, the records' phase bound is within 8 % of it, and the mixed field meets the
    2e-5 relative L2 against the oracle on a strided sample; its largest pixel error is
    also below 2e-5 of the peak."""
    import torch
    wl = near_wide_case()
    b = gpu_trace(wl)
    n = b.shape[0]
    coef = torch.empty(gbd.gbd_project_bytes(n, gbd.GBD_PREC_MIXED), dtype=torch.uint8,
                       device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    gbd.gbd_project(b, n, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED, coef, flag)
    gbd.gbd_sync()
    assert int(flag.item()) & 1 == 0
    # records: tiles of 64 beamlets, fields (i0 j0 a0 p0) (a1u p1u a1v p1v) (auu puu auv puv)
    # (avv pvv . .), SoA inside the tile
    rec = coef.cpu().numpy().view(np.float32).reshape(-1, 4, 64, 4)
    rec = rec.transpose(0, 2, 1, 3).reshape(-1, 16)[:n].astype(np.float64)
    nx, ny = wl.detector.nx, wl.detector.ny
    U = np.maximum(rec[:, 0], nx - 1 - rec[:, 0])
    V = np.maximum(rec[:, 1], ny - 1 - rec[:, 1])
    bound = (np.abs(rec[:, 3]) + np.abs(rec[:, 5]) * U + np.abs(rec[:, 7]) * V +
             np.abs(rec[:, 9]) * U * U + np.abs(rec[:, 11]) * U * V + np.abs(rec[:, 13]) * V * V)
    assert 118.0 < bound.max() <= 128.0, bound.max()
    cols = rows = np.arange(3, nx, 8)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector, cols, rows)
    try:
        if shape is not None:
            gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, shape[0], shape[1], 0, shape[2])
        E = gpu_field(b, wl, gbd.GBD_PREC_MIXED)[np.ix_(rows, cols)]
    finally:
        gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)
    tol = TOL[gbd.GBD_PREC_MIXED]
    assert rel_l2(E, Eo) <= tol, rel_l2(E, Eo)
    peak = np.max(np.abs(Eo))
    assert np.max(np.abs(E - Eo)) <= tol * peak, np.max(np.abs(E - Eo)) / peak


@pytest.mark.parametrize("rows,cols", [(3, 8), (4, 8), (4, 4)])
@pytest.mark.parametrize("name", ["airy_small", "airy_ragged", "defocused", "airy_48"])
def test_row_triples_and_quadruples_match_the_oracle(name, rows, cols):
    """Fields without a uv term: the 3 x 8 and 4 x 8 multi-row kernels (FP32 sums over
    splits of at most 16 tiles) give the oracle's field, and so does the row-pair set that
    runs in their place when a split is longer (airy_48: 1,804 beamlets, 29 tiles in one
    split)."""
    cases = dict(small_cases())
    cases["airy_48"] = W.scaled(W.airy_small(), n_across=48, nx=97, ny=45)
    wl = cases[name]
    b = gpu_trace(wl)
    assert projection_flags(b, wl) & (8 | 16) == 0
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    try:
        for splits in (1, 2, 5):
            gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, rows, cols, splits,
                                    gbd.GBD_SCHEME_ROW_PAIR)
            E = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
            assert rel_l2(E, Eo) <= TOL[gbd.GBD_PREC_MIXED], splits
    finally:
        gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)


@pytest.mark.parametrize("rows,cols", [(3, 8), (4, 8), (4, 4)])
@pytest.mark.parametrize("nx,ny", [(128, 96), (120, 77)])
def test_row_triples_and_quadruples_take_uv_term_fields(rows, cols, nx, ny):
    """The tilted, aberrated optics on a small patch of the focal plane (beamlets ~170
    pixels wide): the field has a uv term and no other flag, so the multi-row kernels'
    instantiation with the per-column row factors P_r = S_r W^r runs (rows 8 r below the
    first as E0 S_r W(tu)^r, W stepped along the row by T^r); the field matches the oracle
    for 1, 2 and 5 splits, on a detector that fills whole thread blocks in neither
    direction as well."""
    wl = W.scaled(W.tilted_zernike(), n_across=16, nx=nx, ny=ny, keep_span=False)
    b = gpu_trace(wl)
    f = projection_flags(b, wl)
    assert f & 8 and not f & (1 | 2 | 4 | 16), f
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    try:
        for splits in (1, 2, 5):
            gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, rows, cols, splits,
                                    gbd.GBD_SCHEME_ROW_PAIR)
            E = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
            assert rel_l2(E, Eo) <= TOL[gbd.GBD_PREC_MIXED], splits
    finally:
        gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)


@pytest.mark.parametrize("rows,cols", [(3, 8), (4, 8), (4, 4)])
def test_multi_row_steep_fields_go_to_the_row_pairs(rows, cols):
    """Pixels 40 times taller than wide on the tilted optics' small patch (beamlets ~170
    pixels wide and ~4 rows tall): a 24-row step's log2 amplitude change exceeds 64 while
    an 8-row step's and the 224-column span's stay within it, so the projection sets the
    cross and multi-row steep bits only; behind the multi-row kernels the row pairs with
    the column factor's update then take the field, and it matches the oracle."""
    import dataclasses
    base = W.scaled(W.tilted_zernike(), n_across=16, nx=128, ny=96, keep_span=False)
    d = base.detector
    wl = dataclasses.replace(base, oracle_stride=None,
                             detector=dataclasses.replace(d, ny=32, pitch_y=40 * d.pitch_x))
    b = gpu_trace(wl)
    assert projection_flags(b, wl) == 8 | 16
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    try:
        for splits in (1, 3):
            gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, rows, cols, splits,
                                    gbd.GBD_SCHEME_ROW_PAIR)
            E = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
            assert rel_l2(E, Eo) <= TOL[gbd.GBD_PREC_MIXED], splits
    finally:
        gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)


def test_column_steep_fields_use_the_general_row_pair_instantiation():
    """Beamlets ~20 pixels wide against a thread's 224-pixel column span: the projection
    flags the amplitude recurrence along rows as unsafe (bit 2) but not the row pairs
    (bit 1); the general instantiation then evaluates each amplitude and the field
    matches the oracle."""
    wl = small_cases()["tilted_zernike_small"]
    b = gpu_trace(wl)
    f = projection_flags(b, wl)
    assert f & 4 and not f & 2
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    for cols in (4, 8):
        try:
            gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, 2, cols, 3, gbd.GBD_SCHEME_ROW_PAIR)
            E = gpu_field(b, wl, gbd.GBD_PREC_MIXED)
        finally:
            gbd.gbd_field_reset_shape(gbd.GBD_PREC_MIXED)
        assert rel_l2(E, Eo) <= TOL[gbd.GBD_PREC_MIXED], cols


@pytest.mark.parametrize("splits", (1, 3))
def test_row_pair_scheme_falls_back_on_steep_beamlets(splits):
    """Beamlets 2.5 pixels wide on a 96-pixel detector: the amplitude changes by more than
    2^64 over 8 rows near the edges, the projection flags it, and the row-pair shape
    evaluates directly instead; the field still matches the oracle."""
    wl = W.Workload("steep", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 4, 1.0, 1.0),
                    W.Detector(96, 96, 1e-5, 1e-5))
    b = gpu_trace(wl)
    assert projection_flags(b, wl) & 2
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    prec = gbd.GBD_PREC_MIXED
    try:
        for cols in (4, 8):
            gbd.gbd_field_set_shape(prec, 2, cols, splits, gbd.GBD_SCHEME_ROW_PAIR)
            E = gpu_field(b, wl, prec)
            assert rel_l2(E, Eo) <= TOL[prec], cols
    finally:
        gbd.gbd_field_reset_shape(prec)


def fallback_cases():
    """Fields that only the fallback launches take, with 51 record tiles: beamlets 64 across
    focused to ~8 pixels on a 512^2 detector of 50 um pixels (steep, wide, column-steep and
    multi-row steep: the direct fallback, every phase reduced) and the 41 lambda F# beamlets
    of near_wide_case on a 704^2 detector (the wide bit alone: the general row pairs)."""
    big = W.airy_large()
    p = big.detector.pitch_x
    return {
        "steep": (W.Workload("steep64", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 64, 1.0, 1.0),
                             W.Detector(512, 512, 5e-5, 5e-5)), 2),
        "wide": (W.Workload("wide704", big.system, W.Pupil(2.4e-3, 64, 1.0, 1.0),
                            W.Detector(704, 704, p, p)), 1),
    }


@pytest.mark.parametrize("shape", [(2, 8), (4, 8), (2, 4)])
@pytest.mark.parametrize("name", ["steep", "wide"])
def test_fallbacks_take_several_splits_per_cta(name, shape):
    """The fallback launches spread their splits in equal shares over about 8 CTAs per SM,
    so with one split per record tile (51) each CTA streams up to six splits in turn, its
    tile barriers' phases carried from one to the next.  The field matches the oracle (on a
    strided sample; the steep field, which lives near the centre, on the central window),
    agrees with 9 splits (one per CTA) to FP32 rounding, and repeats bit for bit."""
    wl, bit = fallback_cases()[name]
    b = gpu_trace(wl)
    f = projection_flags(b, wl)
    assert f & bit and (name == "steep" or f == 1), f
    nx, ny = wl.detector.nx, wl.detector.ny
    # the steep field lives within a few pixels of the centre (5 of a 16-pixel-stride sample
    # above 1e-3 of its peak): its sample is the central 112^2 window
    if name == "steep":
        cols = rows = np.arange(nx // 2 - 56, nx // 2 + 56)
    else:
        cols, rows = np.arange(5, nx, 16), np.arange(3, ny, 16)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector, cols, rows)
    prec = gbd.GBD_PREC_MIXED
    try:
        gbd.gbd_field_set_shape(prec, shape[0], shape[1], 51, gbd.GBD_SCHEME_ROW_PAIR)
        E = gpu_field(b, wl, prec)
        E2 = gpu_field(b, wl, prec)
        gbd.gbd_field_set_shape(prec, shape[0], shape[1], 9, gbd.GBD_SCHEME_ROW_PAIR)
        E9 = gpu_field(b, wl, prec)
    finally:
        gbd.gbd_field_reset_shape(prec)
    assert np.array_equal(E, E2)
    assert rel_l2(E[np.ix_(rows, cols)], Eo) <= TOL[prec]
    assert rel_l2(E, E9) <= 1e-6


def test_autotune_then_parity():
    import torch
    wl = W.airy_small()
    b = gpu_trace(wl)
    prec = gbd.GBD_PREC_MIXED
    ws = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    out = torch.empty((wl.detector.ny, wl.detector.nx), dtype=torch.complex64, device="cuda")
    try:
        r, c, s, ms, scheme = gbd.gbd_autotune_field(b, b.shape[0], wl.system.wavelength,
                                                     wl.detector, prec, ws, out)
        assert ms > 0 and s >= 1
        E = gpu_field(b, wl, prec)
        Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
        assert rel_l2(E, Eo) <= TOL[prec]
    finally:
        gbd.gbd_field_reset_shape(prec)


def test_host_psf_matches_device_path():
    import torch
    wl = W.scaled(W.tilted_zernike(), n_across=16, nx=64, ny=48)
    for prec in PRECS:
        dtype = torch.complex64 if prec == gbd.GBD_PREC_MIXED else torch.complex128
        ws = torch.empty(gbd.gbd_psf_workspace_bytes(wl.pupil, wl.detector, prec),
                         dtype=torch.uint8, device="cuda")
        host = torch.empty((48, 64), dtype=dtype).pin_memory()
        gbd.gbd_psf(wl.system, wl.pupil, wl.pupil.overlap_factor, wl.pupil.waist_ratio,
                    wl.detector, prec, ws, host)
        gbd.gbd_sync()
        E = gpu_field(gpu_trace(wl), wl, prec)
        assert np.array_equal(host.numpy().astype(np.complex128), E)


def test_timeout_is_reported_and_context_survives():
    """A wait limit of one poll makes the producer's wait on busy warps give up: the
    kernel records GBD_ETIMEOUT and exits, and the next call works normally."""
    wl = W.airy_small()
    b = gpu_trace(wl)
    prec = gbd.GBD_PREC_MIXED
    gbd.gbd_field_set_shape(prec, 2, 4, 1)  # every CTA streams all 13 tiles
    try:
        gbd.gbd_set_wait_limit(1)
        gbd.field(b, wl.system.wavelength, wl.detector, prec)
        with pytest.raises(gbd.GbdError) as ei:
            gbd.gbd_sync()
        assert ei.value.status == gbd.GBD_ETIMEOUT
    finally:
        gbd.gbd_set_wait_limit(0)
        gbd.gbd_field_reset_shape(prec)
    E = gpu_field(b, wl, prec)
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    assert rel_l2(E, Eo) <= TOL[prec]


def test_kernel_timing_hooks_count_launches():
    wl = W.airy_small()
    b = gpu_trace(wl)
    gbd.gbd_timing_read()
    gbd.gbd_timing_enable(True)
    try:
        gbd.trace(wl.system, wl.pupil)
        for _ in range(3):
            gbd.field(b, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED)
        gbd.field(b, wl.system.wavelength, wl.detector, gbd.GBD_PREC_F64)
        gbd.gbd_sync()
        t = gbd.gbd_timing_read()
    finally:
        gbd.gbd_timing_enable(False)
    assert t["field_mixed"][1] == 3 and t["field_f64"][1] == 1
    assert t["project"][1] == 4 and t["reduce"][1] == 4 and t["point"][1] == 0
    assert t["trace"][1] == 1
    assert all(t[k][0] > 0 for k in ("field_mixed", "field_f64", "project", "reduce", "trace"))


def test_wide_phase_flag_selects_exact_reduction():
    """On a +-100 lambda F# detector the edge beamlets' phases exceed 128 rad: the
    projection raises the wide-phase flag and the reduced instantiation keeps the mixed
    field within tolerance; on the benchmark workloads (phase bounds up to 101 rad) the
    flag stays clear."""
    import torch
    base = W.airy_small()
    wide = W.Workload("wide", base.system, base.pupil, W.Detector(1024, 1024, 2e-6, 2e-6))
    for wl, expect in ((wide, 1), (W.airy_large(), 0), (W.tilted_zernike(), 0)):
        b = gpu_trace(wl)
        n = b.shape[0]
        coef = torch.empty(gbd.gbd_project_bytes(n, gbd.GBD_PREC_MIXED), dtype=torch.uint8,
                           device="cuda")
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
        gbd.gbd_project(b, n, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED, coef, flag)
        gbd.gbd_sync()
        assert int(flag.item()) & 1 == expect, wl.name
    b = gpu_trace(wide)
    E = gpu_field(b, wide, gbd.GBD_PREC_MIXED)
    idx = np.arange(5, 1024, 33)
    Eo = oracle.field(oracle.trace(wide.system, wide.pupil), wide.system, wide.detector, idx, idx)
    assert rel_l2(E[np.ix_(idx, idx)], Eo) <= TOL[gbd.GBD_PREC_MIXED]


# ------------------------------------------------------------ point evaluation --

def test_point_evaluation_matches_exact_oracle_on_tilted_planes():
    """Every beamlet propagated to every pixel (Sec. 2.2's method) against the oracle's
    exact paraxial propagation; the plane rule differs from it by its method error."""
    for wl in (small_cases()["tilted_zernike_small"], small_cases()["tilted_defocused"]):
        b = gpu_trace(wl)
        E = gbd.field_point(b, wl.system.wavelength, wl.detector)
        gbd.gbd_sync()
        E = E.cpu().numpy()
        o = oracle.trace(wl.system, wl.pupil)
        Ex = oracle.field(o, wl.system, wl.detector, exact=True)
        assert rel_l2(E, Ex) <= 1e-11
        Ep = gpu_field(b, wl, gbd.GBD_PREC_F64)
        assert 0 < rel_l2(Ep, E) < 1e-3


def test_point_equals_plane_on_untilted_plane_and_full_size_subset():
    wl = small_cases()["defocused"]
    b = gpu_trace(wl)
    E = gbd.field_point(b, wl.system.wavelength, wl.detector).cpu().numpy()
    Ep = gpu_field(b, wl, gbd.GBD_PREC_F64)
    assert rel_l2(E, Ep) <= 1e-12
    full = W.tilted_zernike()
    b = gpu_trace(full)
    E = gbd.field_point(b, full.system.wavelength, full.detector)
    gbd.gbd_sync()
    E = E.cpu().numpy()
    cols, rows = W.strided_pixels(full)
    cols, rows = cols[::4], rows[::4]
    Ex = oracle.field(oracle.trace(full.system, full.pupil), full.system, full.detector, cols,
                      rows, exact=True)
    assert rel_l2(E[np.ix_(rows, cols)], Ex) <= 1e-11


# ------------------------------------------------------------ maximum sizes --

@pytest.mark.parametrize("prec", PRECS)
def test_maximum_pupil_grid(prec):
    """4096 beamlets across (13,176,792 beamlets, the largest pupil the ABI accepts) on a
    ragged 72 x 40 detector; the oracle sums every beamlet at a strided 9 x 5 sample."""
    wl = W.Workload("max_pupil", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 4096, 1.5, 1.5),
                    W.Detector(72, 40, 0.8e-6, 0.8e-6))
    b = gpu_trace(wl)
    assert b.shape[0] == oracle.count(4096)
    E = gpu_field(b, wl, prec)
    cols, rows = np.arange(3, 72, 8), np.arange(1, 40, 8)
    o = oracle.trace(wl.system, wl.pupil)
    Eo = oracle.field(o, wl.system, wl.detector, cols, rows)
    assert rel_l2(E[np.ix_(rows, cols)], Eo) <= TOL[prec]


def test_maximum_detector():
    """A 16384 x 16384 detector (the largest the ABI accepts, 2^28 pixels) over +-82 lambda
    F#, so the wide-phase instantiation runs; 52 beamlets; the oracle checks an 11 x 11
    sample across the central +-12 lambda F# that includes the first and last row and
    column."""
    import torch
    n = 16384
    wl = W.Workload("max_det", W.System(1e-6, 0.024, 0.024), W.Pupil(2.4e-3, 8, 1.5, 1.5),
                    W.Detector(n, n, 1e-7, 1e-7))
    b = gpu_trace(wl)
    assert projection_flags(b, wl) & 1
    E = gbd.field(b, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED)
    gbd.gbd_sync()
    idx = np.array([0, 7000, 7600, 7900, 8150, 8192, 8250, 8500, 8800, 9400, n - 1])
    sub = E[torch.as_tensor(idx, device=E.device)][:, torch.as_tensor(idx, device=E.device)]
    sub = sub.cpu().numpy().astype(np.complex128)
    del E
    Eo = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector, idx, idx)
    assert rel_l2(sub, Eo) <= TOL[gbd.GBD_PREC_MIXED]
    assert np.count_nonzero(np.abs(Eo) > 1e-3 * np.abs(Eo).max()) >= 30


# ------------------------------------------------------- streams, threads, graphs --

def test_concurrent_host_threads_on_separate_streams():
    """Two host threads, each with its own stream and workspace, run trace + field at the
    same time on different workloads; each result equals the same call made alone."""
    import threading
    import torch
    cases = [W.airy_small(), W.scaled(W.tilted_zernike(), n_across=24, nx=80, ny=72)]
    alone = []
    for wl in cases:
        b = gpu_trace(wl)
        alone.append(gpu_field(b, wl, gbd.GBD_PREC_MIXED))
    results = [None, None]
    errors = []

    def work(k):
        try:
            wl = cases[k]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(5):
                    b = gbd.trace(wl.system, wl.pupil, stream=s)
                    E = gbd.field(b, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED,
                                  stream=s)
                gbd.gbd_sync(s)
                results[k] = E.cpu().numpy().astype(np.complex128)
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for k in range(2):
        assert np.array_equal(results[k], alone[k])


def test_trace_and_field_replay_from_a_cuda_graph():
    """trace + field captured once into a CUDA graph (torch.cuda.CUDAGraph): with the
    beamlet table and the field zeroed after capture, a replay rebuilds both and equals
    the eager result bit for bit."""
    import torch
    wl = W.airy_small()
    prec = gbd.GBD_PREC_MIXED
    n = gbd.gbd_beamlet_count(wl.pupil)
    beam = torch.empty((n, gbd.BEAMLET_DOUBLES), dtype=torch.float64, device="cuda")
    ws = gbd.workspace(n, wl.detector, prec)
    out = torch.empty((wl.detector.ny, wl.detector.nx), dtype=torch.complex64, device="cuda")
    eager_b = gpu_trace(wl)
    eager = gpu_field(eager_b, wl, prec)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        # one eager pass on the capture stream first (library state, kernel attributes)
        gbd.gbd_trace(wl.system, wl.pupil, wl.pupil.overlap_factor, wl.pupil.waist_ratio,
                      beam, s)
        gbd.gbd_field(beam, n, wl.system.wavelength, wl.detector, prec, ws, out, s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            gbd.gbd_trace(wl.system, wl.pupil, wl.pupil.overlap_factor, wl.pupil.waist_ratio,
                          beam, s)
            gbd.gbd_field(beam, n, wl.system.wavelength, wl.detector, prec, ws, out, s)
    out.zero_()
    beam.zero_()
    g.replay()
    torch.cuda.synchronize()
    gbd.gbd_sync()
    assert np.array_equal(out.cpu().numpy().astype(np.complex128), eager)
