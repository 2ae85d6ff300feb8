"""Host logic of bench.py without a GPU: the replica aggregation over two
gloo ranks, and the reference arm (the oracle) printing its JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_ms = [10.0, 20.0][rank]
    q.put((rank, bench.replica_throughput(dist, t_ms, 1e6, "cpu")))
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    """value = sum of the ranks' particle-steps / the slowest rank's time."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        value, t_max = out[r]
        assert t_max == 20.0
        assert value == pytest.approx(2e6 / 0.020 / 1e6)


def test_single_process_throughput():
    import bench
    value, t = bench.replica_throughput(None, 4.0, 8e5, "cpu")
    assert t == 4.0 and value == pytest.approx(8e5 / 0.004 / 1e6)


def test_reference_arm_prints_its_line():
    """bench.py --impl reference runs the oracle on the host (no GPU needed)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "M particle-steps/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_streaming_roofline_arithmetic():
    """Algorithmic bytes per kernel over its time, against the copy peak."""
    import bench
    kus = {"predict": 10.0, "scan": 4.0, "scatter": 2.0, "gather": 8.0, "momentum": 50.0}
    r = bench.streaming_roofline(kus, 100_000, 50_000, 6800.0)
    assert set(r) == {"predict", "scan", "scatter", "gather"}
    assert r["predict"]["bytes"] == 100_000 * bench.BYTES_PER_PARTICLE["predict"]
    assert r["scan"]["bytes"] == 50_000 * bench.BYTES_PER_CELL_SCAN
    gbs = 100_000 * bench.BYTES_PER_PARTICLE["gather"] / 8e-6 / 1e9
    assert r["gather"]["GB/s"] == round(gbs, 1)
    assert r["gather"]["frac"] == round(gbs / 6800.0, 4)
    assert "momentum" not in r
    assert bench.streaming_roofline({}, 10, 10, 6800.0) == {}


def test_roofline_accounting_follows_the_algorithmic_work():
    """The pair sweeps are bound by FP32 arithmetic and count only the pair
    formulas; the neighbour build is bound by HBM with its own bytes (state,
    list entries, wall tags), never by the 27-cell candidate tests; the step's
    bound uses the pair formulas and 300 state bytes per particle."""
    import bench
    peaks = {"sm_count": 152, "sm_max_mhz": 2070.0, "fp32_tflops": 152 * 128 * 2 * 2070e6 / 1e12,
             "issue_twips": 152 * 4 * 2070e6 / 1e12, "hbm_gbs": 6780.0, "hbm_source": "test"}
    n, ff, fw, act = 80_400, 80_400 * 78.0, 80_400 * 9.0, 15_000.0
    kind, flops = bench.kernel_work("momentum", n, ff, fw, act, 60_000)
    assert kind == "alu" and flops == ff * 50 + fw * 40
    kind, nbytes = bench.kernel_work("neighbors", n, ff, fw, act, 60_000)
    assert kind == "hbm" and nbytes == n * 50 + 4 * (ff + fw + act)
    r = bench.kernel_roofline("neighbors", 0.040, ("hbm", nbytes), peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["frac"] - nbytes / 0.040e-3 / 1e9 / 6780.0) < 1e-12
    s = bench.step_roofline(n, ff, fw, 150.0, peaks)
    want_flops = ff * (36 + 50) + fw * (33 + 40 + 24)
    assert s["flops"] == want_flops and s["bytes"] == 300 * n
    t = max(want_flops / (peaks["fp32_tflops"] * 1e12), 300 * n / (6780e9)) * 1e6
    assert abs(s["frac"] - t / 150.0) < 1e-12


def test_ncu_counters_scale_with_the_workload(monkeypatch):
    """The committed capture is of the 80,400-particle dam break: a line for
    another workload takes its per-launch DRAM bytes and warp instructions
    scaled by the particle count and says so; the capture's own workload takes
    them as recorded."""
    import bench
    rec = {"dram_bytes_per_launch": 1000, "warp_inst_per_launch": 5000.0}
    monkeypatch.setattr(bench, "ncu_traffic", lambda kernel, field="dram_bytes_per_launch": rec[field])
    peaks = {"sm_count": 152, "sm_max_mhz": 2070.0, "fp32_tflops": 80.5, "issue_twips": 1.25856,
             "hbm_gbs": 6780.0, "hbm_source": "test"}
    same = bench.kernel_roofline("neighbors", 0.05, ("hbm", 1e6), peaks)
    assert same["traffic"] == 1000 and same["issue"]["warp_inst_per_launch"] == 5000.0
    assert "traffic_source" not in same
    big = bench.kernel_roofline("neighbors", 0.05, ("hbm", 1e6), peaks, 10 * bench.NCU_CAPTURE_N_FLUID)
    assert big["traffic"] == 10000 and big["issue"]["warp_inst_per_launch"] == 50000.0
    assert "scaled" in big["traffic_source"] and "scaled" in big["issue"]["source"]
