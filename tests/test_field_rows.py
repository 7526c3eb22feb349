"""Row slabs of the field (gbd_field_rows), the building block of pixel sharding.

A slab is evaluated with the whole detector's launch (shape, splits, kernel selection) and
the same thread row blocks, so slabs put together must equal the whole field bit for bit,
for any row boundaries (aligned or not to the kernels' row blocks), both precisions, every
launch shape and the tilted plane's per-pixel carrier.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import shard
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


def cases():
    tz = W.tilted_zernike()
    return {
        "airy_small": W.airy_small(),
        "tilted_zernike_small": W.scaled(tz, n_across=24, nx=80, ny=150),
        "tilted_defocused": W.Workload("tilted_defocused", W.System(0.633e-6, 0.012, 0.0121),
                                       W.Pupil(2.4e-3, 20, 2.0, 1.2),
                                       W.Detector(64, 131, 0.4e-6, 0.5e-6, math.radians(-12),
                                                  math.radians(7))),
        # a uv term and no other flag: the multi-row kernels' uv-term instantiation runs,
        # behind a 4 x 8 pick on 24-row blocks placed at detector rows, so slabs starting at
        # rows 32 or 64 begin 8 or 16 rows into their first block
        "tilted_patch": W.scaled(tz, n_across=16, nx=128, ny=96, keep_span=False),
    }


def boundaries(ny):
    """Row partitions: unaligned cuts, single rows, an empty slab, and the balanced
    partitions of 2, 3 and 8 ranks."""
    out = [[0, 37, 100, ny], [0, 1, 2, 49, 50, ny], [0, 0, 48, 48, ny]]
    for world in (2, 3, 8):
        out.append([a for a, _ in shard.all_slabs(ny, world)] + [ny])
    return [[min(c, ny) for c in cuts] for cuts in out]


def assemble(b, wl, prec, cuts):
    import torch
    parts = []
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        s = gbd.field_rows(b, wl.system.wavelength, wl.detector, r0, r1, prec)
        assert tuple(s.shape) == (r1 - r0, wl.detector.nx)
        parts.append(s)
    gbd.gbd_sync()
    return torch.cat(parts, dim=0)


def shapes(prec):
    D, P = gbd.GBD_SCHEME_DIRECT, gbd.GBD_SCHEME_ROW_PAIR
    if prec == gbd.GBD_PREC_MIXED:
        return [None, (2, 4, D), (1, 4, D), (2, 4, P), (2, 8, P), (3, 8, P), (4, 4, P), (4, 8, P)]
    return [None, (1, 2, D), (2, 2, D), (1, 8, D), (2, 8, D), (1, 32, D), (4, 8, D), (2, 16, D), (8, 4, D)]


def test_tilted_patch_takes_the_uv_term_row_kernels():
    """The tilted patch's flag word is the cross bit alone (its fields go to the multi-row
    kernels' uv-term instantiation, which the slab test below then covers)."""
    import torch
    wl = cases()["tilted_patch"]
    b = gbd.trace(wl.system, wl.pupil)
    n = b.shape[0]
    coef = torch.empty(gbd.gbd_project_bytes(n, gbd.GBD_PREC_MIXED), dtype=torch.uint8,
                       device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    gbd.gbd_project(b, n, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED, coef, flag)
    gbd.gbd_sync()
    assert int(flag.item()) == 8


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(cases()))
def test_slabs_equal_the_whole_field_bit_for_bit(name, prec):
    import torch
    wl = cases()[name]
    b = gbd.trace(wl.system, wl.pupil)
    try:
        for sh in shapes(prec):
            if sh is None:
                gbd.gbd_field_reset_shape(prec)
            else:
                gbd.gbd_field_set_shape(prec, sh[0], sh[1], 3, sh[2])
            whole = gbd.field(b, wl.system.wavelength, wl.detector, prec)
            gbd.gbd_sync()
            for cuts in boundaries(wl.detector.ny):
                got = assemble(b, wl, prec, cuts)
                assert torch.equal(got, whole), (sh, cuts)
    finally:
        gbd.gbd_field_reset_shape(prec)


@pytest.mark.parametrize("prec", PRECS)
def test_slabs_match_the_oracle(prec):
    """The assembled field of the tilted, aberrated case against the oracle (the carrier
    of each slab's rows is that of the whole detector's rows)."""
    wl = cases()["tilted_zernike_small"]
    b = gbd.trace(wl.system, wl.pupil)
    got = assemble(b, wl, prec, [0, 41, 77, wl.detector.ny]).cpu().numpy()
    want = oracle.field(oracle.trace(wl.system, wl.pupil), wl.system, wl.detector)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL[prec]


def test_full_size_airy_large_two_slabs_bit_for_bit():
    """The benchmark's field (51,468 beamlets on 512^2 pixels, its default launch) split
    between two ranks' slabs."""
    import torch
    wl = W.airy_large()
    b = gbd.trace(wl.system, wl.pupil)
    whole = gbd.field(b, wl.system.wavelength, wl.detector, gbd.GBD_PREC_MIXED)
    got = assemble(b, wl, gbd.GBD_PREC_MIXED, [a for a, _ in shard.all_slabs(512, 2)] + [512])
    assert torch.equal(got, whole)


def test_slab_workspace_is_smaller_and_argument_errors():
    import torch
    wl = W.airy_small()
    n = gbd.gbd_beamlet_count(wl.pupil)
    det = wl.detector
    full = gbd.gbd_field_workspace_bytes(n, det, gbd.GBD_PREC_MIXED)
    assert gbd.gbd_field_rows_workspace_bytes(n, det, 0, det.ny, gbd.GBD_PREC_MIXED) == full
    assert gbd.gbd_field_rows_workspace_bytes(n, det, 64, 96, gbd.GBD_PREC_MIXED) < full
    assert gbd.gbd_field_rows_workspace_bytes(n, det, 5, 3, gbd.GBD_PREC_MIXED) == 0
    b = gbd.trace(wl.system, wl.pupil)
    out = torch.empty((4, det.nx), dtype=torch.complex64, device="cuda")
    ws = torch.empty(full, dtype=torch.uint8, device="cuda")
    for r0, r1 in ((-1, 3), (10, det.ny + 1), (9, 8)):
        with pytest.raises(gbd.GbdError):
            gbd.gbd_field_rows(b, n, wl.system.wavelength, det, r0, r1, gbd.GBD_PREC_MIXED, ws,
                               out)
    # an empty range writes nothing
    out.fill_(3.0)
    gbd.gbd_field_rows(b, n, wl.system.wavelength, det, 7, 7, gbd.GBD_PREC_MIXED, ws, out)
    gbd.gbd_sync()
    assert bool((out == 3.0).all())
    # a workspace sized for a small slab is too small for a larger one
    small = gbd.gbd_field_rows_workspace_bytes(n, det, 0, 16, gbd.GBD_PREC_MIXED)
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_field_rows(b, n, wl.system.wavelength, det, 0, 64, gbd.GBD_PREC_MIXED,
                           ws[:small], torch.empty((64, det.nx), dtype=torch.complex64,
                                                  device="cuda"))
    assert ei.value.status == gbd.GBD_ENOMEM
