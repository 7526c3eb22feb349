#!/usr/bin/env python
"""Throughput of plane-evaluation Gaussian beamlet decomposition on GB300.

One step = one pass of the hot path over the 512 x 512-pixel, 51,468-beamlet Airy workload
(2.4 mm pupil, lambda 1 um, F/10, 256 beamlets across, +-20 lambda F#): gbd_trace
(decomposition + differential trace) and gbd_field (per-beamlet projection, per-pixel
evaluation, coherent sum) in the mixed FP32/FP64 path.  The metric is beamlet-pixel
evaluations per second.  Also reported: the FP64 path on the same workload, the error of
both against the FP64 CPU oracle on a pixel sample, an end-to-end number through the
host-buffer call gbd_psf, the field kernel's fraction of the MUFU-pipe roofline and the
oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica (the workload does not need a
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("beamlet·pixel evals/s on 1 GB300, mixed vs FP64 path, at stated error vs FP64 "
          "oracle")
UNIT = "evals/s"
# MUFU (XU pipe) results per clock per SM on GB300: sin and cos at 16 (the CUDA
# programming guide's rate for these functions), ex2 at 32 (Blackwell Ultra doubles the
# exponential rate; the live probe measures both).  SM count and maximum SM clock.
MUFU_EX2_PER_CLK_SM = 32
MUFU_SINCOS_PER_CLK_SM = 16
GB300_SMS = 152
GB300_MAX_MHZ = 2070.0
# Per-launch DRAM bytes of the multi-row field kernel on airy_large from one ncu capture
# (the field_mixed_rows_kernel summary under profiles/), and its issued warp-instructions
# per 32 evaluations.  The reads are the record tiles; the writes are the summed field:
# the kernel sums its split partials itself in L2 and drops their lines, so its DRAM
# traffic does not grow with the split count.
FIELD_MIXED_NCU = [
    {"kernel": "field_mixed_rows_kernel<4, 4> (4x4 row quadruples)", "read": 3.3344e6,
     "write": 2.884352e6, "splits": 90, "rows": 4, "cols": 4, "scheme": 1,
     "inst_per_32_evals": 6.81, "fma_pipe_active": 0.675},
    {"kernel": "field_mixed_rows_kernel<4, 8> (4x8 row quadruples, packed FP32x2)",
     "read": 3.364864e6, "write": 4.082944e6, "splits": 90, "rows": 4, "cols": 8, "scheme": 1,
     "inst_per_32_evals": 4.38, "fma_pipe_active": 0.730},
]
ISSUE_PER_CLK_SM = 4  # warp-instructions issued per clock and SM (one per sub-partition)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=2,
                    help="timed runs of the 1024-instance parameter sweep (0 = skip)")
    ap.add_argument("--sweep-instances", type=int, default=1024,
                    help="instances of the sweep (a seeded draw from the same distributions; "
                         "fewer only for small profiling runs)")
    ap.add_argument("--no-point", action="store_true",
                    help="skip the plane- versus point-evaluation comparison")
    ap.add_argument("--shape", default="",
                    help="fixed mixed launch shape 'rows,cols,splits[,scheme]' instead of the "
                         "autotuner's pick (scheme 1 = row pairs)")
    ap.add_argument("--no-telescope", action="store_true",
                    help="skip the App. B telescope (conic-mirror trace + field) line")
    ap.add_argument("--no-tilted", action="store_true",
                    help="skip the tilted, aberrated system's mixed field line")
    ap.add_argument("--no-telescope-sweep", action="store_true",
                    help="skip the 1024-instance sweep and the search on the App. B telescope")
    ap.add_argument("--no-sharding", action="store_true",
                    help="skip the pixel-sharded field (row slabs + gather)")
    ap.add_argument("--no-truncated", action="store_true",
                    help="skip the truncated-beamlet fields")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the surrogate-guided search versus grid and random search")
    return ap.parse_args()


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_block(wl, nb):
    det = wl.detector
    return {
        "workload": (f"{wl.name}: {nb} beamlets x {det.nx}x{det.ny} pixels, lambda "
                     f"{wl.system.wavelength * 1e6:g} um, F/{wl.f_number:g}, "
                     f"{wl.pupil.n_across} beamlets across, OF {wl.pupil.overlap_factor}"),
        "n_beamlets": nb,
        "n_pixels": det.nx * det.ny,
        "evals_per_step": nb * det.nx * det.ny,
        "l2": "flushed between timed steps (256 MB write); step inputs < L2",
        "parallelism": "replicas (no data-path collective)",
    }


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", gpu_index], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.windows = []

    def mark(self):
        return time.time()

    def add_window(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        import datetime
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[5:]))
            except Exception:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if any(a - 0.06 <= r[0] <= b + 0.06 for a, b in self.windows)]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mhz = sorted(r[1] for r in use)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for r in use:
            flags = r[3]
            for name, flag in zip(names, flags[1:5]):
                if flag.lower() in ("active", "0x1", "1"):
                    reasons.add(name)
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted(reasons), "samples": len(use),
                "samples_in_timed_region": len(inside)}


def ncu_capture(tuned):
    """The ncu record of the launch shape that ran, or None."""
    for n in FIELD_MIXED_NCU:
        if (tuned[0], tuned[1], tuned[4]) == (n["rows"], n["cols"], n["scheme"]):
            return n
    return None


def traffic_bytes(tuned):
    """Per-launch DRAM bytes of the captured kernel (records read, field written; neither
    depends on the split count)."""
    n = ncu_capture(tuned)
    if n is None:
        return None
    return n["read"] + n["write"]


def mufu_mix(rows: int = 1, cols: int = 0, scheme: int = 0, cross: bool = False):
    """MUFU operations per beamlet-pixel evaluation (ex2, and sin = cos) of a launch shape.
    Direct scheme: one ex2, sin and cos per evaluation.  Row pairs on 2 x cols pixels, per
    beamlet and block: cols + 1 sin/cos pairs (the first row and the exact row-step
    factor) and 4 ex2 (that factor, and the first row's amplitude, its column ratio and the
    ratio's ratio); the second row comes from multiplies on the FMA pipe.  Without a uv term
    (cross = False, the bench's workloads) the step factor is the same on every column and
    is formed once per beamlet and warp of 32 blocks: 3 ex2 and cols sin/cos pairs per block,
    plus that factor's ex2 and sin/cos pair per warp.  Row triples or
    quadruples on rows x cols pixels (no uv term): cols sin/cos pairs and 2 ex2 per block,
    plus per beamlet and warp of 32 blocks the shared 3 ex2 and two sin/cos pairs of the
    row terms (the step factors R and K, the amplitude ratio's ratio)."""
    if not scheme or not cols:
        return 1.0, 1.0
    if rows in (3, 4):
        px = float(rows * cols)
        return 2.0 / px + 3.0 / (32 * px), cols / px + 2.0 / (32 * px)
    if not cross:
        px = 2.0 * cols
        return 3.0 / px + 1.0 / (32 * px), cols / px + 1.0 / (32 * px)
    return 4.0 / (2 * cols), (cols + 1) / (2.0 * cols)


def peak_evals_const(cols: int = 0, rows: int = 2, cross: bool = False) -> float:
    """MUFU-bound beamlet-pixel evaluations/s of a GB300 at its maximum clock: the direct
    scheme (cols = 0), or the row-pair / row-triple scheme on rows x cols pixels."""
    n_ex2, n_sc = mufu_mix(rows, cols, 1 if cols else 0, cross)
    return GB300_SMS * GB300_MAX_MHZ * 1e6 / (n_ex2 / MUFU_EX2_PER_CLK_SM +
                                              2.0 * n_sc / MUFU_SINCOS_PER_CLK_SM)


def gpu_index_for_smi(local: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local] if vis else str(local)


# ------------------------------------------------------------- CPU oracle --

def oracle_sample_rate(wl, seconds: float, rows_hint=None):
    """Oracle evals/s on a strided row sample sized to about `seconds` of CPU time."""
    import numpy as np

    import oracle
    o = oracle.trace(wl.system, wl.pupil)
    nb = o.shape[0]
    cols = np.arange(wl.detector.nx)
    if rows_hint is None:
        t0 = time.perf_counter()
        oracle.field(o, wl.system, wl.detector, cols, [wl.detector.ny // 2])
        t1 = time.perf_counter() - t0
        n_rows = int(max(1, min(wl.detector.ny, seconds / max(t1, 1e-6))))
    else:
        n_rows = rows_hint
    rows = np.linspace(0, wl.detector.ny - 1, n_rows).round().astype(int)
    t0 = time.perf_counter()
    E = oracle.field(o, wl.system, wl.detector, cols, rows)
    dt = time.perf_counter() - t0
    evals = nb * cols.size * rows.size
    return {"value": evals / dt, "seconds": dt, "evals": evals, "rows": rows, "cols": cols,
            "field": E, "cores": oracle.threads(), "nb": nb}


# ------------------------------------------------------------------- ours --

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2404_12454_gb300 import gbd
    from paper_2404_12454_gb300 import workloads as W

    # one build per node (the in-tree objects are shared), then every rank loads it
    if local == 0:
        __graft_entry__.build()
    barrier(world)
    if local != 0:
        __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.airy_large()
    sysm, pupil, det = wl.system, wl.pupil, wl.detector
    nb = gbd.gbd_beamlet_count(pupil)
    npix = det.nx * det.ny
    evals = nb * npix
    MIX, F64 = gbd.GBD_PREC_MIXED, gbd.GBD_PREC_F64

    beam = torch.empty((nb, 36), dtype=torch.float64, device=dev)
    ws = {p: torch.empty(max(256, gbd.gbd_field_workspace_bytes(nb, det, p)), dtype=torch.uint8,
                         device=dev) for p in (MIX, F64)}
    out = {MIX: torch.empty((det.ny, det.nx), dtype=torch.complex64, device=dev),
           F64: torch.empty((det.ny, det.nx), dtype=torch.complex128, device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(prec):
        gbd.gbd_trace(sysm, pupil, pupil.overlap_factor, pupil.waist_ratio, beam, stream)
        gbd.gbd_field(beam, nb, sysm.wavelength, det, prec, ws[prec], out[prec], stream)

    def timed(prec, k, clocks=None):
        times = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec)
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    clocks = ClockSampler(gpu_index_for_smi(local))
    # the library's autotuner picks the launch shape (pixels per thread, beamlet splits,
    # scheme) unless --shape fixes it
    gbd.gbd_trace(sysm, pupil, pupil.overlap_factor, pupil.waist_ratio, beam, stream)
    if args.shape:
        v = [int(x) for x in args.shape.split(",")]
        gbd.gbd_field_set_shape(MIX, v[0], v[1], v[2], v[3] if len(v) > 3 else 0)
        r_, c_, s_, k_ = gbd.gbd_field_get_shape(MIX, nb, det)
        tuned = (r_, c_, s_, 0.0, k_)
    else:
        tune_ws = torch.empty(320 << 20, dtype=torch.uint8, device=dev)
        tuned = gbd.gbd_autotune_field(beam, nb, sysm.wavelength, det, MIX, tune_ws, out[MIX],
                                       stream)
        del tune_ws
    # the split count the launches use: whole tiles per split (93 requested -> 90 for
    # 805 tiles)
    n_tiles_mix = (nb + 63) // 64
    tps_mix = -(-n_tiles_mix // max(1, min(tuned[2], n_tiles_mix)))
    tuned = (tuned[0], tuned[1], -(-n_tiles_mix // tps_mix), tuned[3], tuned[4])
    ws[MIX] = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nb, det, MIX)), dtype=torch.uint8,
                          device=dev)
    for _ in range(args.warmup):
        step(MIX)
    gbd.gbd_sync(stream)

    # ---- mixed path, K timed steps
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    gbd.gbd_timing_read()
    gbd.gbd_timing_enable(True)
    t0 = time.time()
    ms = timed(MIX, args.steps)
    t1 = time.time()
    gbd.gbd_timing_enable(False)
    clocks.add_window(t0, t1)
    gbd.gbd_sync(stream)
    torch.cuda.synchronize()
    barrier(world)
    kt = gbd.gbd_timing_read()
    total_ms = allreduce_max(world, sum(ms))
    ms_per_step = total_ms / args.steps
    value = world * evals * args.steps / (total_ms * 1e-3)
    E_mix = out[MIX].cpu().numpy().astype(np.complex128)

    # ---- the direct scheme (every pixel by ex2 + sin + cos) on the same step, for
    # comparison with the scheme the autotuner picked; then the picked shape is restored
    direct = None
    if tuned[4]:
        gbd.gbd_field_set_shape(MIX, 2, 4, 0, gbd.GBD_SCHEME_DIRECT)
        ws_d = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nb, det, MIX)),
                           dtype=torch.uint8, device=dev)
        ws_keep, ws[MIX] = ws[MIX], ws_d
        timed(MIX, 2)
        gbd.gbd_timing_read()
        gbd.gbd_timing_enable(True)
        md = timed(MIX, 3)
        gbd.gbd_timing_enable(False)
        gbd.gbd_sync(stream)
        kd = gbd.gbd_timing_read()["field_mixed"]
        kd_s = kd[0] / max(kd[1], 1) * 1e-3
        direct = {"shape": "2x4 direct", "value": evals * len(md) / (sum(md) * 1e-3),
                  "unit": UNIT, "kernel_ms": kd_s * 1e3,
                  "frac_of_mufu_peak": evals / kd_s / peak_evals_const()}
        ws[MIX] = ws_keep
        del ws_d
        gbd.gbd_field_set_shape(MIX, tuned[0], tuned[1], tuned[2], tuned[4])

    # ---- FP64 path on the same workload
    f64 = None
    if args.fp64_steps > 0:
        # the FP64 path's row-segment shape, picked by one timed run each (the library's
        # autotuner would spend tens of seconds on this 0.4 s kernel)
        best64 = None
        for shp in ((1, 32), (4, 8), (8, 4)):
            gbd.gbd_field_set_shape(F64, shp[0], shp[1], 0)
            ws[F64] = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nb, det, F64)),
                                  dtype=torch.uint8, device=dev)
            t = timed(F64, 1)[0]
            if best64 is None or t < best64[1]:
                best64 = (shp, t)
        gbd.gbd_field_set_shape(F64, best64[0][0], best64[0][1], 0)
        ws[F64] = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nb, det, F64)),
                              dtype=torch.uint8, device=dev)
        step(F64)
        gbd.gbd_sync(stream)
        t0 = time.time()
        ms64 = timed(F64, args.fp64_steps)
        clocks.add_window(t0, time.time())
        total64 = allreduce_max(world, sum(ms64))
        v64 = world * evals * args.fp64_steps / (total64 * 1e-3)
        E_64 = out[F64].cpu().numpy()
        f64 = {"value": v64, "unit": UNIT, "ms_per_step": total64 / args.fp64_steps,
               "steps": args.fp64_steps, "mixed_speedup": value / v64,
               "shape": f"{best64[0][0]}x{best64[0][1]} row segments",
               "mixed_vs_fp64_rel_l2": float(np.linalg.norm(E_mix - E_64) / np.linalg.norm(E_64))}

    # ---- end to end: host-side parameters in, host field out, through gbd_psf
    ws_psf = torch.empty(gbd.gbd_psf_workspace_bytes(pupil, det, MIX), dtype=torch.uint8, device=dev)
    host = torch.empty((det.ny, det.nx), dtype=torch.complex64).pin_memory()

    def psf_step():
        gbd.gbd_psf(sysm, pupil, pupil.overlap_factor, pupil.waist_ratio, det, MIX, ws_psf, host,
                    stream)
        gbd.gbd_sync(stream)

    for _ in range(2):
        psf_step()
    barrier(world)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        psf_step()
        e2e_t.append(time.perf_counter() - a)
    e2e_total = allreduce_max(world, sum(e2e_t))
    gbd_system_bytes = 4 * 8 + 4 + 64 * 4 + 64 * 8 + 4  # gbd_system as passed (with padding)
    e2e = {"value": world * evals * args.steps / e2e_total, "unit": UNIT,
           "h2d_bytes_per_step": gbd_system_bytes + 16 + 40,
           "d2h_bytes_per_step": npix * 8,
           "api": "gbd_psf (host parameters -> pinned host complex64 field)",
           # host-clock spread of the steps (the value is their sum: a host stall counts)
           "step_ms_median": float(np.median(e2e_t)) * 1e3,
           "step_ms_max": float(np.max(e2e_t)) * 1e3}

    # ---- batched parameter sweep: 1024 uneven instances in one persistent launch, replayed
    # as a CUDA graph on its own stream
    sweep = None
    if args.sweep_steps > 0:
        sw = W.sweep(n_instances=args.sweep_instances)
        sstream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(sstream):
            plan = gbd.sweep_plan(sw, stream=sstream)
            plan.run(stream=sstream, graph=True)
            sstream.synchronize()
            sms = []
            t0 = time.time()
            for _ in range(args.sweep_steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(sstream)
                plan.run(stream=sstream, graph=True)
                b.record(sstream)
                sms.append((a, b))
            sstream.synchronize()
            clocks.add_window(t0, time.time())
        gbd.gbd_sync(sstream)
        sweep_ms = allreduce_max(world, sum(x.elapsed_time(y) for x, y in sms))
        sv = world * plan.evals * args.sweep_steps / (sweep_ms * 1e-3)
        sc = plan.scores.cpu().numpy()
        sweep = {"value": sv, "unit": UNIT, "ms_per_sweep": sweep_ms / args.sweep_steps,
                 "instances": plan.n, "beamlets": plan.beamlets, "evals_per_sweep": plan.evals,
                 "work_items": plan.items,
                 "shape": "3x8 row triples (library default)",
                 "frac_of_mufu_peak": sv / world / peak_evals_const(8, rows=3),
                 "frac_of_direct_scheme_mufu_peak": sv / world / peak_evals_const(),
                 "graph": True, "score_range": [float(sc.min()), float(sc.max())],
                 "workload": f"{plan.n} instances, airy_small optics, OF~U[1,3], WR~U[0.8,3], "
                             "N~U{16..256}, 256x256 pixels +-5 lambda F#"}
        plan.close()

    # ---- the same 1024 seeded draws traced by real rays through the App. B telescope (the
    # optics Sec. 6 searches), image plane at the system's least-RMS focus
    sweep_tel = None
    if args.sweep_steps > 0 and not args.no_telescope_sweep:
        tsw = W.telescope_sweep(n_instances=args.sweep_instances)
        sstream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(sstream):
            tplan = gbd.sweep_plan(tsw, stream=sstream)
            tplan.run(stream=sstream, graph=True)
            sstream.synchronize()
            tms = []
            t0 = time.time()
            for _ in range(args.sweep_steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(sstream)
                tplan.run(stream=sstream, graph=True)
                b.record(sstream)
                tms.append((a, b))
            sstream.synchronize()
            clocks.add_window(t0, time.time())
        gbd.gbd_sync(sstream)
        tsweep_ms = allreduce_max(world, sum(x.elapsed_time(y) for x, y in tms))
        tsc = tplan.scores.cpu().numpy()
        sweep_tel = {"value": world * tplan.evals * args.sweep_steps / (tsweep_ms * 1e-3),
                     "unit": UNIT, "ms_per_sweep": tsweep_ms / args.sweep_steps,
                     "instances": tplan.n, "beamlets": tplan.beamlets,
                     "evals_per_sweep": tplan.evals, "graph": True,
                     "score_range": [float(tsc.min()), float(tsc.max())],
                     "workload": f"{tplan.n} instances (the seeded draws above) traced through "
                                 "the App. B telescope (real rays, two conics), 256x256 pixels "
                                 "of 2.8 mas at its least-RMS focus"}
        tplan.close()

    # ---- one field over the ranks by detector rows (gbd_field_rows + all_gather); on one
    # GPU the slabs of a 2- and an 8-way split run one after another (no collective)
    sharding = None
    if not args.no_sharding:
        from paper_2404_12454_gb300 import shard

        def slab_ms(r0, r1, reps=5):
            wsb = torch.empty(max(256, gbd.gbd_field_rows_workspace_bytes(nb, det, r0, r1, MIX)),
                              dtype=torch.uint8, device=dev)
            o = torch.empty((max(r1 - r0, 1), det.nx), dtype=torch.complex64, device=dev)
            gbd.gbd_field_rows(beam, nb, sysm.wavelength, det, r0, r1, MIX, wsb, o, stream)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                gbd.gbd_field_rows(beam, nb, sysm.wavelength, det, r0, r1, MIX, wsb, o, stream)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        gbd.gbd_trace(sysm, pupil, pupil.overlap_factor, pupil.waist_ratio, beam, stream)
        whole = slab_ms(0, det.ny)
        sharding = {"whole_field_ms": whole,
                    "note": "beamlet table replicated, rows split, one all_gather; slabs are "
                            "bit-identical to the whole field's rows"}
        for split in (2, 8):
            per = [slab_ms(a, b) for a, b in shard.all_slabs(det.ny, split)]
            sharding[f"slabs_{split}_ms"] = per
            sharding[f"slabs_{split}_efficiency_bound"] = whole / (split * max(per))
        if world > 1:
            r0, r1 = shard.slab_bounds(det.ny, world, rank)
            times = []
            for k in range(args.warmup + args.steps):
                barrier(world)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                gbd.gbd_trace(sysm, pupil, pupil.overlap_factor, pupil.waist_ratio, beam, stream)
                shard.field_sharded(beam, sysm.wavelength, det, MIX, stream=stream)
                torch.cuda.synchronize()
                if k >= args.warmup:
                    times.append(time.perf_counter() - t0)
            t_max = allreduce_max(world, sum(times))
            sharding.update({"ranks": world, "ms_per_field": t_max / args.steps * 1e3,
                             "value": evals * args.steps / t_max, "unit": UNIT,
                             "scaling": "strong"})

    # ---- plane evaluation versus point evaluation (Sec. 2.2's method) on the tilted,
    # aberrated workload at 256^2 pixels over the same span, both FP64
    point = None
    if not args.no_point:
        tz = W.scaled(W.tilted_zernike(), nx=256, ny=256)
        bt = gbd.trace(tz.system, tz.pupil, stream=stream)
        nbt = bt.shape[0]
        ev = nbt * 256 * 256
        Ep = gbd.field(bt, tz.system.wavelength, tz.detector, F64, stream=stream)
        Eq = gbd.field_point(bt, tz.system.wavelength, tz.detector, stream=stream)
        gbd.gbd_sync(stream)
        wsq = torch.empty(max(256, gbd.gbd_field_point_workspace_bytes(nbt, tz.detector)),
                          dtype=torch.uint8, device=dev)
        wsp = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nbt, tz.detector, F64)),
                          dtype=torch.uint8, device=dev)
        def ms_of(fn):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b2 = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(2):
                fn()
            b2.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b2) / 2

        # the plane rule on its fastest FP64 shape for this field (it has a uv term, so the
        # row-factor tables of the multi-row shapes do not apply)
        t = {"plane": math.inf}
        plane_shape = None
        for shp in ((1, 32), (4, 8), (8, 4)):
            gbd.gbd_field_set_shape(F64, shp[0], shp[1], 0)
            wsp = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nbt, tz.detector, F64)),
                              dtype=torch.uint8, device=dev)
            tp = ms_of(lambda: gbd.gbd_field(bt, nbt, tz.system.wavelength, tz.detector, F64,
                                             wsp, Ep, stream))
            if tp < t["plane"]:
                t["plane"], plane_shape = tp, shp
        gbd.gbd_field_set_shape(F64, plane_shape[0], plane_shape[1], 0)
        wsp = torch.empty(max(256, gbd.gbd_field_workspace_bytes(nbt, tz.detector, F64)),
                          dtype=torch.uint8, device=dev)
        gbd.gbd_field(bt, nbt, tz.system.wavelength, tz.detector, F64, wsp, Ep, stream)
        t["point"] = ms_of(lambda: gbd.gbd_field_point(bt, nbt, tz.system.wavelength,
                                                       tz.detector, wsq, Eq, stream))
        gbd.gbd_sync(stream)
        Epn, Eqn = Ep.cpu().numpy(), Eq.cpu().numpy()
        point = {"workload": f"tilted_zernike optics, {nbt} beamlets x 256x256 pixels (same span), FP64",
                 "plane_shape": f"{plane_shape[0]}x{plane_shape[1]}",
                 "plane_evals_per_s": ev / (t["plane"] * 1e-3),
                 "point_evals_per_s": ev / (t["point"] * 1e-3),
                 "plane_over_point_speedup": t["point"] / t["plane"],
                 "plane_vs_point_rel_l2": float(np.linalg.norm(Epn - Eqn) / np.linalg.norm(Eqn))}

    # ---- the App. B telescope: real-ray trace through its two conic mirrors, then the
    # mixed-precision plane evaluation, 256 beamlets across on 512^2 pixels of 2.8 mas
    telescope = None
    if not args.no_telescope:
        msys, tpup, tdet = W.hst_rc(n_across=256, npix=512)
        nbr = gbd.gbd_beamlet_count(tpup)
        br = torch.empty((nbr, gbd.BEAMLET_DOUBLES), dtype=torch.float64, device=dev)
        wsr = gbd.workspace(nbr, tdet, MIX, dev)
        Er = torch.empty((tdet.ny, tdet.nx), dtype=torch.complex64, device=dev)

        def rc_step():
            gbd.gbd_trace_mirrors(msys, tpup, tpup.overlap_factor, tpup.waist_ratio, br, stream)
            gbd.gbd_field(br, nbr, msys.wavelength, tdet, MIX, wsr, Er, stream)
        for _ in range(3):
            rc_step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b2 = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            rc_step()
        b2.record(stream)
        torch.cuda.synchronize()
        gbd.gbd_sync(stream)
        rc_ms = a.elapsed_time(b2) / 3
        airy_peak = math.pi * W.HST_DIAMETER[0] ** 2 / (4.0 * msys.wavelength * W.HST_EFL)
        telescope = {"workload": f"App. B Ritchey-Chretien telescope, {nbr} beamlets x "
                                 f"{tdet.nx}x{tdet.ny} pixels of 2.8 mas, real-ray trace + mixed field",
                     "ms_per_psf": rc_ms, "value": nbr * tdet.nx * tdet.ny / (rc_ms * 1e-3),
                     "unit": UNIT,
                     "centre_over_airy_peak": float(abs(Er[tdet.ny // 2, tdet.nx // 2].item())
                                                    / airy_peak)}

    # ---- the tilted, aberrated system (Zernike plate, detector tilted 10 deg / 5 deg):
    # trace + mixed field at 1024^2 pixels, the default shape (a field with a uv term, so
    # the row triples with per-column row factors run behind the 4 x 8 pick); parity on it
    # is a test case
    tilted = None
    if not args.no_tilted:
        twl = W.tilted_zernike()
        tsys = twl.system
        ntb = gbd.gbd_beamlet_count(twl.pupil)
        bt = torch.empty((ntb, gbd.BEAMLET_DOUBLES), dtype=torch.float64, device=dev)
        wst = gbd.workspace(ntb, twl.detector, MIX, dev)
        Et = torch.empty((twl.detector.ny, twl.detector.nx), dtype=torch.complex64, device=dev)

        def tz_step():
            gbd.gbd_trace(tsys, twl.pupil, twl.pupil.overlap_factor, twl.pupil.waist_ratio, bt,
                          stream)
            gbd.gbd_field(bt, ntb, tsys.wavelength, twl.detector, MIX, wst, Et, stream)
        for _ in range(3):
            tz_step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b2 = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            tz_step()
        b2.record(stream)
        torch.cuda.synchronize()
        gbd.gbd_sync(stream)
        tz_ms = a.elapsed_time(b2) / 3
        tr, tc, ts_, tsch = gbd.gbd_field_get_shape(MIX, ntb, twl.detector)
        tilted = {"workload": f"tilted_zernike: {ntb} beamlets x {twl.detector.nx}x"
                              f"{twl.detector.ny} pixels, Noll 4-15 plate, detector tilted "
                              "10 deg about x and 5 deg about y",
                  "ms_per_field": tz_ms,
                  "value": ntb * twl.detector.nx * twl.detector.ny / (tz_ms * 1e-3),
                  "unit": UNIT, "shape": f"{tr}x{tc}, {ts_} splits, scheme {tsch}"}

    # ---- truncated beamlets (edge beamlets cut by the aperture's tangent half-plane): the
    # distance to the exact hard-aperture focal field on the small Airy workload, and the
    # cost of the cut field next to the plain one on both Airy workloads
    truncated = None
    if not args.no_truncated:
        from scipy.special import j1 as bessel_j1

        def timed_ms(fn, reps=5):
            fn()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        truncated = {}
        for name in ("airy_small", "airy_large"):
            tw = W.by_name(name)
            bp = gbd.trace(tw.system, tw.pupil, stream=stream)
            bc, ne = gbd.trace_truncated(tw.system, tw.pupil, stream=stream)
            out_p = torch.empty((tw.detector.ny, tw.detector.nx), dtype=torch.complex64, device=dev)
            out_c = torch.empty_like(out_p)
            wsp = gbd.workspace(bp.shape[0], tw.detector, MIX)
            wsc = torch.empty(gbd.gbd_field_truncated_workspace_bytes(bc.shape[0], ne, tw.detector,
                                                                      MIX),
                              dtype=torch.uint8, device=dev)
            t_plain = timed_ms(lambda: gbd.gbd_field(bp, bp.shape[0], tw.system.wavelength,
                                                     tw.detector, MIX, wsp, out_p, stream))
            t_cut = timed_ms(lambda: gbd.gbd_field_truncated(bc, bc.shape[0], ne,
                                                             tw.system.wavelength, tw.detector,
                                                             MIX, wsc, out_c, stream))
            gbd.gbd_sync(stream)
            ent = {"beamlets": int(bc.shape[0]), "edge_beamlets": ne,
                   "plain_beamlets": int(bp.shape[0]), "plain_ms": t_plain, "truncated_ms": t_cut}
            if name == "airy_small":
                det_s = tw.detector
                lam_s, f_s, R_s = tw.system.wavelength, tw.system.focal_length, tw.pupil.diameter / 2
                k_s = 2 * math.pi / lam_s
                xs = (np.arange(det_s.nx) - det_s.nx // 2) * det_s.pitch_x
                Xs, Ys = np.meshgrid(xs, xs)
                rs = np.hypot(Xs, Ys)
                us = k_s * R_s * rs / f_s
                safe = np.where(us == 0, 1.0, us)
                exact = ((1j / (lam_s * f_s)) * np.exp(-1j * k_s * rs * rs / (2 * f_s)) * math.pi
                         * R_s * R_s * np.where(us == 0, 1.0, 2 * bessel_j1(safe) / safe))
                for key, o in (("plain_vs_hard_aperture_rel_l2", out_p),
                               ("truncated_vs_hard_aperture_rel_l2", out_c)):
                    e = o.cpu().numpy().astype(np.complex128)
                    ent[key] = float(np.linalg.norm(e - exact) / np.linalg.norm(exact))
            truncated[name] = ent

    # ---- surrogate-guided search versus the reference grid and random search
    surrogate = None
    if not args.no_surrogate:
        from paper_2404_12454_gb300 import surrogate as S
        t0 = time.perf_counter()
        grid = S.grid_search()
        t_grid = time.perf_counter() - t0
        target = 1.01 * grid.best[1]
        t0 = time.perf_counter()
        sur = S.surrogate_search(rounds=3)
        t_sur = time.perf_counter() - t0
        n_sur = sur.evals_to_reach(target)
        rnd = S.random_search(budget=len(sur.scores))
        step_us = S.time_training_device(1024, 100)  # CUDA events around one 100-step call
        fit_us = S.time_training(1024, 100)  # wall time of MLP.fit (host copies included)
        # ablation over 8 seeds, both searches starting from the same 32 random draws and
        # spending 32 evaluations per round: the contract's 1 % target (flat here: any
        # 256-across set with OF < 1.45 meets it) and a 0.01 % target
        ablation = {}
        for label, frac in (("within_1pct", 1e-2), ("within_0.01pct", 1e-4)):
            r = S.compare_with_random((1.0 + frac) * grid.best[1], seeds=range(1, 9))
            cap = 1260

            def mean_evals(v):
                return float(np.mean([cap if x is None else x for x in v]))
            ablation[label] = {"surrogate_evals": r["surrogate"], "random_evals": r["random"],
                               "surrogate_mean": mean_evals(r["surrogate"]),
                               "random_mean_capped_at_1260": mean_evals(r["random"])}
        # the same search on the App. B telescope (real-ray traced instances): the 1 % window
        # there is OF below ~1.15 at 256 across
        sur_tel = None
        if not args.no_telescope_sweep:
            optics = W.telescope_sweep_from_params
            tgrid = S.grid_search(optics=optics)
            sur_tel = {"grid_evals": len(tgrid.scores), "grid_best": tgrid.best[1],
                       "grid_best_params": list(tgrid.best[0])}
            for label, frac in (("within_1pct", 1e-2), ("within_0.1pct", 1e-3)):
                r = S.compare_with_random((1.0 + frac) * tgrid.best[1], seeds=range(8),
                                          optics=optics)
                sur_tel[label] = {"surrogate_evals": r["surrogate"], "random_evals": r["random"],
                                  "surrogate_mean": mean_evals(r["surrogate"]),
                                  "random_mean_capped_at_1260": mean_evals(r["random"])}
        surrogate = {"grid_evals": len(grid.scores), "grid_best": grid.best[1],
                     "grid_best_params": list(grid.best[0]), "grid_seconds": t_grid,
                     "surrogate_evals_to_1pct": n_sur, "surrogate_best": sur.best[1],
                     "surrogate_best_params": list(sur.best[0]), "surrogate_seconds": t_sur,
                     "surrogate_evals": len(sur.scores),
                     "median_proposal_score": float(np.median(sur.scores[128:])),
                     "random_best_same_budget": rnd.best[1],
                     "median_random_score": float(np.median(rnd.scores[128:])),
                     "mlp_train_step_us_batch1024": step_us,
                     "mlp_fit_us_per_step_batch1024": fit_us,
                     "ablation_8_seeds_init32": ablation, "telescope": sur_tel}

    clk = clocks.stop()

    # ---- roofline of the dominant kernel (mixed field kernel, MUFU pipe), with the MUFU
    # operations per evaluation of the scheme that ran (mufu_mix)
    kms, kn = kt["field_mixed"]
    k_avg_s = (kms / max(kn, 1)) * 1e-3
    probes = gbd.gbd_probe_peaks()
    n_ex2, n_sc = mufu_mix(tuned[0], tuned[1], tuned[4])
    clk_per_eval = n_ex2 / MUFU_EX2_PER_CLK_SM + 2.0 * n_sc / MUFU_SINCOS_PER_CLK_SM
    peak_direct = GB300_SMS * GB300_MAX_MHZ * 1e6 / (1.0 / MUFU_EX2_PER_CLK_SM +
                                                    2.0 / MUFU_SINCOS_PER_CLK_SM)
    peak_evals = GB300_SMS * GB300_MAX_MHZ * 1e6 / clk_per_eval
    probe_peak = 1.0 / (n_ex2 / probes["ex2"] + n_sc / probes["sin"] + n_sc / probes["cos"])
    achieved = evals / k_avg_s
    roofline = {
        "bound": "alu",
        "pipe": (f"MUFU (XU): {n_ex2:.4g} ex2 + {n_sc:.4g} sin + {n_sc:.4g} cos per "
                 "beamlet-pixel (scheme " + ("row_pair" if tuned[4] else "direct") + ")"),
        "achieved": achieved / 1e9, "peak": peak_evals / 1e9, "unit": "Geval/s",
        "frac": achieved / peak_evals,
        "traffic": traffic_bytes(tuned),
        "traffic_source": (("ncu dram__bytes_read.sum + dram__bytes_write.sum of one capture of "
                            f"{ncu_capture(tuned)['kernel']} at {ncu_capture(tuned)['splits']} "
                            "splits (the kernel sums its split partials in L2)")
                           if ncu_capture(tuned) else "no ncu capture of this launch shape"),
        "peak_source": (f"derived: {GB300_SMS} SMs x {GB300_MAX_MHZ:g} MHz / ({n_ex2:.4g}/"
                        f"{MUFU_EX2_PER_CLK_SM} + {2 * n_sc:.4g}/{MUFU_SINCOS_PER_CLK_SM}) clk "
                        "per evaluation"),
        "kernel": ("field_mixed_rows_kernel" if tuned[4] and tuned[0] in (3, 4)
                   else "field_mixed_pair_smem_kernel" if tuned[4] and tuned[1] >= 8
                   else "field_mixed_kernel") + f" ({tuned[0]}x{tuned[1]}, {tuned[2]} splits)",
        "kernel_ms_avg": k_avg_s * 1e3, "launches": kn,
        "mufu_gops": (n_ex2 + 2.0 * n_sc) * achieved / 1e9,
        "direct_scheme_peak": peak_direct / 1e9,
        "frac_of_direct_scheme_peak": achieved / peak_direct,
        "probe_ops_per_s": probes,
        "probe_peak_evals_per_s": probe_peak,
        "frac_of_probe_peak": achieved / probe_peak,
    }
    # The multi-row kernels need so few MUFU operations that instruction issue binds first:
    # the issue-slot ceiling for the captured kernel's instruction count per evaluation.
    cap = ncu_capture(tuned)
    if cap is not None:
        ipe = cap["inst_per_32_evals"] / 32.0
        issue_peak = GB300_SMS * GB300_MAX_MHZ * 1e6 * ISSUE_PER_CLK_SM / ipe
        roofline["issue_bound"] = {
            "warp_instructions_per_32_evals": cap["inst_per_32_evals"],
            "peak": issue_peak / 1e9, "unit": "Geval/s", "frac": achieved / issue_peak,
            "source": ("ncu smsp__inst_executed.sum of the capture; 152 SMs x 4 issue slots "
                       "x 2070 MHz")}
        # what binds the packed kernels: the FMA-heavy pipe (the packed FP32x2 operations
        # and the phase FMAs); its busy fraction over the captured launch
        roofline["fma_pipe"] = {
            "active_frac": cap["fma_pipe_active"],
            "source": "ncu sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active of the capture"}

    # ---- error and CPU baseline (rank 0, one GPU)
    cpu = None
    error = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample_rate(wl, args.cpu_seconds)
        rows, cols = r["rows"], r["cols"]
        Eo = r["field"]
        error["mixed_vs_oracle_rel_l2"] = float(
            np.linalg.norm(E_mix[np.ix_(rows, cols)] - Eo) / np.linalg.norm(Eo))
        if f64 is not None:
            error["fp64_vs_oracle_rel_l2"] = float(
                np.linalg.norm(E_64[np.ix_(rows, cols)] - Eo) / np.linalg.norm(Eo))
        cpu = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": f"{rows.size} of {det.ny} rows x {cols.size} columns x {r['nb']} beamlets "
                         f"({r['evals']:.3g} evals, {r['seconds']:.1f} s, FP64 C + OpenMP)"}

    # trace, projection, split reduction, and the field kernels of the shape: the
    # instantiation the flag word selects plus the others, which return at once (direct:
    # 2; row pairs on 2 or 4 columns: 3; on 8 columns: 4; row triples / quadruples: their
    # two instantiations, without and with a uv term, and 3 row-pair launches behind them,
    # or the 8-column pairs alone (4) when a split holds more than 16 tiles)
    tiles = -(-nb // 64)
    tiles_per_split = -(-tiles // max(1, tuned[2]))
    if not tuned[4]:
        field_launches = 2
    elif tuned[0] >= 3:
        field_launches = 5 if tiles_per_split <= 16 else 4
    elif tuned[1] >= 8:
        field_launches = 4
    else:
        field_launches = 3
    launches_per_step = 3 + field_launches
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": ("mixed: FP64 per-beamlet trace/projection, FP32 per-pixel phase with MUFU "
                      "ex2/sin/cos" + ((" (the rows 8, 16, 24 below each evaluated row by FP32 "
                                        "complex products with exact row-step factors; FP32 "
                                        "sums over splits of at most 1,024 beamlets)")
                                       if tuned[4] and tuned[0] >= 3 else
                                       (" (second row of each pair by an FP32 complex row-step "
                                        "factor; TwoSum across 64-beamlet tiles)")
                                       if tuned[4] else " (TwoSum across 64-beamlet tiles)")
                      + ", splits summed with compensation (Neumaier)"),
        "data": "synthetic (ideal F/10 lens standing in for the paper's traced telescope)",
        "config": config_block(wl, nb), "clocks": clk, "e2e": e2e, "fp64_path": f64,
        "direct_scheme": direct,
        "autotuned_shape": {"rows_per_thread": tuned[0], "cols_per_thread": tuned[1],
                            "splits": tuned[2], "ms": tuned[3],
                            "scheme": "row_pair" if tuned[4] else "direct",
                            "fixed_by_flag": bool(args.shape)},
        "sweep": sweep, "sweep_telescope": sweep_tel, "surrogate": surrogate,
        "point_evaluation": point, "telescope": telescope, "tilted": tilted,
        "pixel_sharding": sharding, "truncated": truncated,
        "error": error, "roofline": roofline, "cpu_baseline": cpu,
        "gpu_launches": launches_per_step * args.steps,
        "kernel_ms": {k: (v[0] / max(v[1], 1)) for k, v in kt.items()},
    }
    line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def summary(line: dict) -> dict:
    """The headline figures of the line's blocks in a few short keys, printed last (a reader
    of the line's tail sees them without parsing the blocks)."""
    def g(*path, digits=4):
        v = line
        for p in path:
            if not isinstance(v, dict) or p not in v:
                return None
            v = v[p]
        return float(f"{v:.{digits}g}") if isinstance(v, (int, float)) else v

    return {
        "mixed_evals_per_s": g("value"), "ms_per_step": g("ms_per_step"),
        "roofline_frac": g("roofline", "frac"), "issue_frac": g("roofline", "issue_bound", "frac"),
        "fp64_evals_per_s": g("fp64_path", "value"), "mixed_over_fp64": g("fp64_path", "mixed_speedup"),
        "err_mixed": g("error", "mixed_vs_oracle_rel_l2", digits=3),
        "err_fp64": g("error", "fp64_vs_oracle_rel_l2", digits=3),
        "e2e_evals_per_s": g("e2e", "value"),
        "sweep_ms": g("sweep", "ms_per_sweep"), "sweep_evals_per_s": g("sweep", "value"),
        "sweep_telescope_ms": g("sweep_telescope", "ms_per_sweep"),
        "sweep_telescope_evals_per_s": g("sweep_telescope", "value"),
        "tilted_evals_per_s": g("tilted", "value"), "telescope_psf_ms": g("telescope", "ms_per_psf"),
        "plane_over_point": g("point_evaluation", "plane_over_point_speedup"),
        "search_lens_0.01pct_evals_sur_vs_rnd": [
            g("surrogate", "ablation_8_seeds_init32", "within_0.01pct", "surrogate_mean"),
            g("surrogate", "ablation_8_seeds_init32", "within_0.01pct", "random_mean_capped_at_1260")],
        "search_telescope_1pct_evals_sur_vs_rnd": [
            g("surrogate", "telescope", "within_1pct", "surrogate_mean"),
            g("surrogate", "telescope", "within_1pct", "random_mean_capped_at_1260")],
        "search_telescope_0.1pct_evals_sur_vs_rnd": [
            g("surrogate", "telescope", "within_0.1pct", "surrogate_mean"),
            g("surrogate", "telescope", "within_0.1pct", "random_mean_capped_at_1260")],
        "mlp_step_us": g("surrogate", "mlp_train_step_us_batch1024"),
        "sharding_8_slab_efficiency_bound": g("pixel_sharding", "slabs_8_efficiency_bound"),
        "truncated_small_err_plain_vs_cut": [
            g("truncated", "airy_small", "plain_vs_hard_aperture_rel_l2", digits=3),
            g("truncated", "airy_small", "truncated_vs_hard_aperture_rel_l2", digits=3)],
        "truncated_large_ms_plain_vs_cut": [g("truncated", "airy_large", "plain_ms"),
                                            g("truncated", "airy_large", "truncated_ms")],
        "gpu_launches": line.get("gpu_launches"),
    }


# -------------------------------------------------------------- reference --

def run_reference(args, world, rank, local):
    """The FP64 CPU oracle as it stands, timed on the host cores, one bounded sample of the
    same workload per step."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2404_12454_gb300 import workloads as W
    import oracle.build as ob
    ob.build()
    wl = W.airy_large()
    o = oracle.trace(wl.system, wl.pupil)
    nb = o.shape[0]
    cols = np.arange(wl.detector.nx)
    rows_per_step = 2
    times = []
    for s in range(args.warmup + args.steps):
        rows = [(37 * s + 11 * q) % wl.detector.ny for q in range(rows_per_step)]
        t0 = time.perf_counter()
        oracle.field(o, wl.system, wl.detector, cols, rows)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    evals = nb * cols.size * rows_per_step
    total = sum(times)
    value = evals * len(times) / total
    cpu = {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
           "sample": f"{rows_per_step} rows x {cols.size} columns x {nb} beamlets per step"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(wl, nb), "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank, local)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
