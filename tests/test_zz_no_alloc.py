"""gbd_field_noalloc: the field entry point for callers that may not allocate device memory
(a plugin whose host application owns every device allocation, a real-time loop with
memory fixed at start-up).  Its scratch is a fixed array inside the library, so the test
calls it twice in a row through the C ABI and checks each result against gbd_field (the
entry point with a caller workspace) within the parity tolerances of the other tests.

Kept in a file that pytest collects last, so a run that stops at the first failure has
run every other test before this one.
"""
import numpy as np
import pytest

from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {gbd.GBD_PREC_F64: 1e-11, gbd.GBD_PREC_MIXED: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_12454_gb300 import build
    build.build()
    import torch
    torch.cuda.init()


def _cases():
    return [W.airy_small(), W.scaled(W.tilted_zernike(), n_across=40, nx=200, ny=136),
            W.airy_large()]


@pytest.mark.parametrize("prec", [gbd.GBD_PREC_F64, gbd.GBD_PREC_MIXED])
def test_noalloc_matches_workspace_entry_point_twice(prec):
    import torch
    for wl in _cases():
        b = gbd.trace(wl.system, wl.pupil)
        ref = gbd.field(b, wl.system.wavelength, wl.detector, prec)
        gbd.gbd_sync()
        ref = ref.cpu().numpy().astype(np.complex128)
        dtype = torch.complex64 if prec == gbd.GBD_PREC_MIXED else torch.complex128
        for _ in range(2):
            out = torch.full((wl.detector.ny, wl.detector.nx), 3.0, dtype=dtype, device="cuda")
            gbd.gbd_field_noalloc(b, b.shape[0], wl.system.wavelength, wl.detector, prec, out)
            gbd.gbd_sync()
            got = out.cpu().numpy().astype(np.complex128)
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            assert err <= TOL[prec], (wl.name, err)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    wl = W.airy_small()
    b = gbd.trace(wl.system, wl.pupil)
    big = W.Detector(2048, 2048, 1e-7, 1e-7)  # one partial field alone is 64 MiB
    out = torch.empty((2048, 2048), dtype=torch.complex64, device="cuda")
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_field_noalloc(b, b.shape[0], wl.system.wavelength, big, gbd.GBD_PREC_MIXED, out)
    assert ei.value.status == gbd.GBD_EINVAL
    assert "scratch" in str(ei.value)
    gbd.gbd_sync()
