"""Host-side logic of bench.py without a GPU: the replica timing across ranks (gloo,
world size 2), the reference arm (the FP64 oracle timed on the host cores) and the
roofline arithmetic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_init(None)
    bench.barrier(w)
    # every rank reports its own elapsed time; the line uses the slowest rank's
    got = bench.allreduce_max(w, 1.5 + r)
    q.put((r, w, got))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "8"))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "evals/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True


def test_roofline_arithmetic():
    """The MUFU operations per evaluation behind the bench line's roofline: the direct
    scheme's 3, the row pairs' (cols + 1) sin/cos pairs and 4 ex2 per 2 x cols block (3 ex2
    and cols pairs plus the warp's share without a uv term), the multi-row kernels' cols
    pairs and 2 ex2 per block plus the warp's share; and the peaks derived from 152 SMs at
    2070 MHz with 32 ex2 and 16 sin/cos per clock and SM."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.mufu_mix() == (1.0, 1.0)
    assert bench.peak_evals_const() == pytest.approx(152 * 2.07e9 / (1 / 32 + 2 / 16))
    ex2, sc = bench.mufu_mix(2, 8, 1, cross=True)
    assert (ex2, sc) == pytest.approx((0.25, 9 / 16))
    ex2, sc = bench.mufu_mix(2, 8, 1)
    assert (ex2, sc) == pytest.approx((3 / 16 + 1 / 512, 8 / 16 + 1 / 512))
    ex2, sc = bench.mufu_mix(3, 8, 1)
    assert (ex2, sc) == pytest.approx((2 / 24 + 3 / 768, 8 / 24 + 2 / 768))
    ex2, sc = bench.mufu_mix(4, 4, 1)
    assert (ex2, sc) == pytest.approx((2 / 16 + 3 / 512, 4 / 16 + 2 / 512))
    # fewer MUFU operations per evaluation, a higher ceiling
    assert bench.peak_evals_const(8, rows=3) > bench.peak_evals_const(8) > bench.peak_evals_const()
    # every recorded ncu capture matches its own shape; the multi-row kernel sums its split
    # partials in L2, so its traffic does not depend on the split count
    for cap in bench.FIELD_MIXED_NCU:
        tuned = (cap["rows"], cap["cols"], cap["splits"], 0.0, cap["scheme"])
        assert bench.ncu_capture(tuned) is cap
        assert bench.traffic_bytes(tuned) == pytest.approx(cap["read"] + cap["write"])
        doubled = (cap["rows"], cap["cols"], 2 * cap["splits"], 0.0, cap["scheme"])
        assert bench.traffic_bytes(doubled) == pytest.approx(cap["read"] + cap["write"])
    assert bench.traffic_bytes((1, 4, 10, 0.0, 0)) is None
