"""Host-side logic of bench.py (no GPU): the traffic table lookup, the
roofline arithmetic, the replica aggregation and the reference arm's JSON
line (the FP64 oracle on a small crop of the same workload)."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2412_12734_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


@pytest.mark.parametrize("kernel", sorted(bench.TRAFFIC))
def test_traffic_is_reported_only_for_captured_sources_and_configs(kernel, monkeypatch):
    t = bench.TRAFFIC[kernel]
    cfg, value = t["measured"][0]
    argv = ["--workload", cfg["workload"], "--tex-n", str(cfg["tex_n"]), "--tile", str(cfg["tile"])]
    if "batch" in cfg:
        argv += ["--batch", str(cfg["batch"])]
    if "batch_fwd" in cfg:
        argv += ["--batch-fwd", str(cfg["batch_fwd"])]
    if "ppt" in cfg:
        argv += ["--ppt", str(cfg["ppt"])]
    args = bench.parse(argv)
    expect = value if _digest(t["files"]) == t["sha256_16"] else None
    assert bench.measured_traffic(kernel, args) == expect
    # another launch configuration, a subset of the views, or other sources: no figure
    other = bench.parse(argv + ["--tile", "8"])
    assert bench.measured_traffic(kernel, other) is None
    assert bench.measured_traffic(kernel, bench.parse(argv + ["--views", "2"])) is None
    monkeypatch.setitem(bench.TRAFFIC, kernel, dict(t, sha256_16="0" * 16))
    assert bench.measured_traffic(kernel, args) is None


def test_forward_traffic_follows_the_forward_batch_depth():
    t = bench.TRAFFIC["render_fwd"]
    if _digest(t["files"]) != t["sha256_16"]:
        pytest.skip("forward sources changed since the capture")
    cfg, value = t["measured"][0]
    base = ["--workload", cfg["workload"], "--tex-n", str(cfg["tex_n"]), "--tile", str(cfg["tile"])]
    # --batch alone sets both passes; --batch-fwd overrides the forward's
    assert bench.measured_traffic("render_fwd", bench.parse(base + ["--batch", str(cfg["batch_fwd"])])) == value
    assert bench.measured_traffic("render_fwd", bench.parse(base + ["--batch", "8", "--batch-fwd",
                                                                    str(cfg["batch_fwd"])])) == value
    assert bench.measured_traffic("render_fwd", bench.parse(base + ["--batch", str(cfg["batch_fwd"]),
                                                                    "--batch-fwd", "128"])) is None


def test_roofline_line_arithmetic():
    st = {"pairs_bwd": 1.0e9, "contributing_bwd": 0.5e9, "pairs_fwd": 2.0e9, "blended_fwd": 1.0e9}
    r = bench.roofline_line("render_bwd", {"render_bwd": 40.0, "render_fwd": 10.0}, st, {"sm_mhz": 2000.0}, 4.0e9)
    flops = 30 * 1.0e9 + 200 * 0.5e9
    assert r["achieved"] == pytest.approx(flops / 0.040 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert (r["bound"], r["unit"], r["traffic"], r["kernel"]) == ("alu", "TFLOP/s", 4.0e9, "render_bwd")
    f = bench.roofline_line("render_fwd", {"render_fwd": 10.0}, st, {"sm_mhz": None})
    assert f["achieved"] == pytest.approx((30 * 2.0e9 + 61 * 1.0e9) / 0.010 / 1e12)
    assert f["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS_AT_MAX)
    assert f["traffic"] is None


def test_single_rank_aggregate():
    ms, value = bench.aggregate(18_086_400, 50.0, 1)
    assert ms == 50.0
    assert value == pytest.approx(18_086_400 / 0.050 / 1e6)


def test_reference_arm_prints_one_contract_line():
    """`--impl reference` times the FP64 oracle on a bounded crop and prints
    the contract's line on the same metric, unit and workload label."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--crop", "16"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Mpixel/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    wl = bench.make_workload(bench.parse([]))
    assert d["config"]["workload"] == bench.workload_label(bench.parse([]), wl)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "16x16" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
