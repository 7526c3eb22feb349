"""The C-ABI library builds, loads and exports every symbol include/gbd.h declares; the
host-side argument checks reject bad input before any launch (no GPU needed)."""
import ctypes
import math
import os
import re

import pytest

from paper_2404_12454_gb300 import build as gbuild
from paper_2404_12454_gb300 import gbd
from paper_2404_12454_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_]\w*[\s\*]+\**(gbd_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gbd.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # and the binding covers every declaration under the same name
    missing = [n for n in names if n not in gbd._SIGS]
    assert not missing, missing


def test_version_and_beamlet_count(lib):
    assert "sm_103a" in gbd.gbd_version()
    for n, expected in ((1, 1), (2, 4), (16, 208), (32, 812), (64, 3228), (128, 12892), (256, 51468)):
        assert gbd.gbd_beamlet_count(W.Pupil(2.4e-3, n, 1.5, 1.5)) == expected
    assert lib.gbd_beamlet_count(None) == -1
    assert gbd.gbd_beamlet_count(W.Pupil(2.4e-3, 0, 1.5, 1.5)) == -1


def test_beamlet_count_equals_brute_force(lib):
    """The per-row closed count (integer square roots) against the plain double loop over
    the grid's inside-test (2i-(N-1))^2 + (2j-(N-1))^2 <= N^2, for every N up to 600."""
    for n in range(1, 601):
        want = 0
        for j in range(n):
            b = 2 * j - (n - 1)
            a = [2 * i - (n - 1) for i in range(n)]
            want += sum(1 for x in a if x * x + b * b <= n * n)
        assert gbd.gbd_beamlet_count(W.Pupil(2.4e-3, n, 1.5, 1.5)) == want, n


def _einval(call):
    with pytest.raises(gbd.GbdError) as ei:
        call()
    assert ei.value.status in (gbd.GBD_EINVAL, gbd.GBD_ENOMEM)
    return ei.value.status


def test_trace_rejects_bad_arguments(lib):
    wl = W.airy_small()
    null = None

    class T:  # stands in for a tensor; never dereferenced: validation fails first
        shape = (10 ** 6, 36)

        def data_ptr(self):
            return 16

    good_sys, good_pup = wl.system, wl.pupil
    bad = [
        (W.System(-1e-6, 0.024, 0.024), good_pup),
        (W.System(float("nan"), 0.024, 0.024), good_pup),
        (W.System(1e-6, 0.0, 0.024), good_pup),
        (W.System(1e-6, 0.024, -1.0), good_pup),
        (W.System(1e-6, 0.024, 0.024, (70,), (1e-7,), 1e-3), good_pup),
        (W.System(1e-6, 0.024, 0.024, (4,), (1e-7,), 0.0), good_pup),
        (good_sys, W.Pupil(-1.0, 32, 1.5, 1.5)),
        (good_sys, W.Pupil(2.4e-3, 5000, 1.5, 1.5)),
    ]
    for s, p in bad:
        assert _einval(lambda: gbd.gbd_trace(s, p, 1.5, 1.5, T())) == gbd.GBD_EINVAL
    assert _einval(lambda: gbd.gbd_trace(good_sys, good_pup, 0.0, 1.5, T())) == gbd.GBD_EINVAL
    assert _einval(lambda: gbd.gbd_trace(good_sys, good_pup, 1.5, -1.0, T())) == gbd.GBD_EINVAL

    class Small(T):
        shape = (5, 36)
    assert _einval(lambda: gbd.gbd_trace(good_sys, good_pup, 1.5, 1.5, Small())) == gbd.GBD_ENOMEM
    assert "capacity" in lib.gbd_last_error().decode()


def test_trace_mirrors_rejects_bad_arguments(lib):
    msys, pupil, _ = W.hst_rc(n_across=16)

    class T:
        shape = (10 ** 6, 36)

        def data_ptr(self):
            return 16

    def with_(**kw):
        d = dict(wavelength=msys.wavelength, radius=msys.radius, conic=msys.conic,
                 spacing=msys.spacing, diameter=msys.diameter, pupil_offset=msys.pupil_offset)
        d.update(kw)
        return W.MirrorSystem(**d)

    bad = [
        with_(wavelength=0.0),
        with_(pupil_offset=0.0),
        with_(radius=(), conic=(), spacing=(), diameter=()),
        with_(radius=(0.0, 1.358)),
        with_(radius=(float("inf"), 1.358)),
        with_(spacing=(-4.9, 0.0)),
        with_(conic=(float("nan"), -1.5)),
    ]
    for m in bad:
        assert _einval(lambda: gbd.gbd_trace_mirrors(m, pupil, 1.5, 1.0, T())) == gbd.GBD_EINVAL
    assert _einval(lambda: gbd.gbd_trace_mirrors(msys, pupil, 0.0, 1.0, T())) == gbd.GBD_EINVAL
    assert _einval(lambda: gbd.gbd_trace_mirrors(msys, W.Pupil(-1.0, 16, 1.5, 1.0), 1.5, 1.0,
                                                 T())) == gbd.GBD_EINVAL

    class Small(T):
        shape = (5, 36)
    assert _einval(lambda: gbd.gbd_trace_mirrors(msys, pupil, 1.5, 1.0, Small())) == gbd.GBD_ENOMEM
    with pytest.raises(ValueError):
        gbd.make_mirror_system(with_(radius=(-1.0,) * 5, conic=(0.0,) * 5, spacing=(1.0,) * 5))


def test_field_rejects_bad_arguments(lib):
    det = W.airy_small().detector

    class T:
        def __init__(self, addr=256, n=1 << 20):
            self.addr, self.n = addr, n

        def data_ptr(self):
            return self.addr

        def numel(self):
            return self.n

        def element_size(self):
            return 1

    cases = [
        dict(detector=W.Detector(0, 10, 1e-6, 1e-6)),
        dict(detector=W.Detector(10, 10, -1e-6, 1e-6)),
        dict(detector=W.Detector(10, 10, 1e-6, 1e-6, 2.0, 0.0)),
        dict(precision=7),
        dict(wavelength=0.0),
        dict(n=-1),
        dict(ws=T(addr=300)),  # misaligned workspace
        dict(out=T(addr=8)),   # misaligned output
    ]
    for c in cases:
        args = dict(beam=T(), n=10, wavelength=1e-6, detector=det, precision=gbd.GBD_PREC_MIXED,
                    ws=T(), out=T())
        args.update(c)
        st = _einval(lambda: gbd.gbd_field(args["beam"], args["n"], args["wavelength"],
                                           args["detector"], args["precision"], args["ws"],
                                           args["out"]))
        assert st == gbd.GBD_EINVAL
    with pytest.raises(gbd.GbdError):
        gbd.gbd_field_set_shape(gbd.GBD_PREC_MIXED, 3, 3)


def test_mlp_rejects_bad_arguments(lib):
    class T:
        def __init__(self, addr=256, n=1 << 26, rows=64):
            self.addr, self.n, self.shape = addr, n, (rows, 3)

        def data_ptr(self):
            return self.addr

        def numel(self):
            return self.n

    B = 64
    need = gbd.gbd_mlp_workspace_bytes(B)
    # six transposed operands in two BF16 parts, a_4 and d_1 in FP32, y and dL/dy
    assert need >= 12 * 128 * B * 2 + 2 * 128 * B * 4 + 2 * B * 4
    assert gbd.gbd_mlp_workspace_bytes(0) == 0
    base = dict(master=T(), weights=T(), m=T(), v=T(), x=T(), target=T(), lr=1e-3, b1=0.9,
                b2=0.999, eps=1e-8, first=1, steps=3, loss=T(), ws=T(n=need))
    cases = [
        (dict(master=None), gbd.GBD_EINVAL),
        (dict(weights=T(addr=264)), gbd.GBD_EINVAL),   # weights not 16-byte aligned
        (dict(ws=T(addr=272, n=need)), gbd.GBD_EINVAL),  # workspace not 256-byte aligned
        (dict(ws=T(n=need - 1)), gbd.GBD_ENOMEM),
        (dict(x=T(rows=0)), gbd.GBD_EINVAL),
        (dict(x=T(rows=(1 << 20) + 1)), gbd.GBD_EINVAL),
        (dict(steps=-1), gbd.GBD_EINVAL),
        (dict(first=0), gbd.GBD_EINVAL),
        (dict(first=2 ** 31 - 2, steps=5), gbd.GBD_EINVAL),
        (dict(lr=0.0), gbd.GBD_EINVAL),
        (dict(b1=1.0), gbd.GBD_EINVAL),
        (dict(eps=-1.0), gbd.GBD_EINVAL),
    ]
    for c, want in cases:
        a = dict(base)
        a.update(c)
        if a["x"].shape[0] != B and "ws" not in c:
            a["ws"] = T(n=max(256, gbd.gbd_mlp_workspace_bytes(a["x"].shape[0])))
        with pytest.raises(gbd.GbdError) as ei:
            gbd.gbd_mlp_train(a["master"], a["weights"], a["m"], a["v"], a["x"], a["target"],
                              a["lr"], a["b1"], a["b2"], a["eps"], a["first"], a["steps"],
                              a["loss"], a["ws"])
        assert ei.value.status == want, (c, ei.value.status)
    with pytest.raises(gbd.GbdError):
        gbd.gbd_mlp_forward(T(addr=258), T(), T())
    with pytest.raises(gbd.GbdError):
        gbd.gbd_mlp_adam(T(), T(), T(), T(), T(), 1e-3, 0.9, 0.999, 1e-8, 0)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gbd, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gbd, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        gbd.lib()


def test_sweep_plan_layout_on_the_host(lib):
    """gbd_sweep_plan_create is host-only: the 1024-instance sweep's work list for the
    default shape (row triples, 256 x 24-pixel items: 11 per instance on 256^2 pixels) and
    for row pairs (256 x 16: 16 per instance) and direct 1 x 4 blocks (128 x 8: 64), the
    same evaluation and beamlet totals (the sum over instances of beamlets x pixels), and
    unsupported shapes rejected before anything is allocated on a device."""
    sw = W.sweep()
    n, a, b, c = gbd._instance_arrays(sw.n_across, sw.overlap_factor, sw.waist_ratio)
    counts = [gbd.gbd_beamlet_count(sw.pupil(k)) for k in range(n)]
    npix = sw.detector.nx * sw.detector.ny

    def create(shape):
        p = ctypes.c_void_p()
        sh = gbd.gbd_shape(shape[0], shape[1], 1, 0.0, shape[2]) if shape else None
        st = lib.gbd_sweep_plan_create(ctypes.byref(gbd.make_system(sw.system)),
                                       float(sw.diameter), a, b, c, n,
                                       ctypes.byref(gbd.make_detector(sw.detector)),
                                       ctypes.byref(sh) if sh else None, ctypes.byref(p))
        return st, p

    for shape, per_instance in ((None, 11), ((3, 8, 1), 11), ((2, 8, 1), 16), ((1, 4, 0), 64)):
        st, p = create(shape)
        assert st == gbd.GBD_OK, shape
        try:
            ev, nb, items = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int32()
            assert lib.gbd_sweep_info(p, ctypes.byref(ev), ctypes.byref(nb),
                                      ctypes.byref(items)) == gbd.GBD_OK
            assert items.value == n * per_instance, shape
            assert nb.value == sum(counts)
            assert ev.value == float(sum(counts) * npix)
            assert lib.gbd_sweep_workspace_bytes(p) > 64 * nb.value  # the records at least
        finally:
            lib.gbd_sweep_plan_destroy(p)
    for shape in ((3, 4, 1), (4, 4, 1), (2, 8, 0), (3, 3, 1)):
        st, p = create(shape)
        assert st == gbd.GBD_EINVAL, shape


@pytest.mark.parametrize("N,OF,margin", [(32, 1.5, 3.0), (17, 2.2, 2.0), (4, 1.5, 3.0),
                                         (64, 1.0, 0.0), (9, 1.2, 1.0)])
def test_truncated_count_matches_oracle(lib, N, OF, margin):
    """Host-side count of the truncated decomposition (whole + edge beamlets) against the
    oracle's enumeration (N = 4 with margin 3: every beamlet is an edge beamlet)."""
    import oracle
    pupil = W.Pupil(2.4e-3, N, OF, 1.0)
    sysm = W.System(1e-6, 0.024, 0.024)
    recs, dist, ne = oracle.trace_truncated(sysm, pupil, margin=margin)
    assert gbd.gbd_truncated_count(pupil, OF, margin) == (recs.shape[0], ne)
    assert gbd.gbd_truncated_count(pupil, OF, -1.0)[0] == -1
    assert gbd.gbd_truncated_count(pupil, -1.0, 3.0)[0] == -1
