"""bench.py's host-side pieces on the CPU: the roofline arithmetic of each
step kernel and the reference arm's JSON line (the oracle timed on the host
cores), so that a change to either shows up without a GPU."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PK = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1500.0, "sm_max_mhz": 2000.0}
L2PK = {"scatter_reductions_per_s": 2e11, "gather_loads_per_s": 3e11}
D = (32, 64, 64, 1)


def test_adam_roofline_counts_34_bytes_per_visited_parameter(bench):
    avg = {"adam": 0.05}
    r = bench.roofline_of("adam", avg, "fp16", PK, "measured", 1 << 18, 1_000_000, 0, D, 16, 2, L2PK)
    assert r["algorithmic_bytes_per_launch"] == 34_000_000
    assert r["achieved"] == pytest.approx(34e6 / 0.05e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["params_visited_per_launch"] == 1_000_000
    r32 = bench.roofline_of("adam", avg, "fp32", PK, "measured", 1 << 18, 1_000_000, 0, D, 16, 2, L2PK)
    assert r32["algorithmic_bytes_per_launch"] == 32_000_000


def test_mlp_roofline_is_the_l2_scatter(bench):
    batch = 1 << 18
    avg = {"mlp": 0.15}
    r = bench.roofline_of("mlp", avg, "fp16", PK, "measured", batch, 1, 0, D, 16, 2, L2PK)
    assert r["kernel"] == "k_mlp_tc" and r["bound"] == "l2" and r["unit"] == "GB/s"
    # algorithmic bytes: the scatter's 8 corners x L x F FP32 reductions per point
    assert r["algorithmic_bytes_per_launch"] == batch * 8 * 16 * 2 * 4
    assert r["achieved"] == pytest.approx(batch * 1024 / 0.15e-3 / 1e9)
    assert r["peak"] == pytest.approx(2e11 * 16 / 1e9)  # the measured reduction rate x 16 B
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["hbm"]["algorithmic_bytes_per_launch"] == batch * (2 * 32 + 4 + 8 * 16 * 2 * 4)
    assert r["hbm"]["peak"] == 6000.0
    flops = 2 * batch * (32 * 64 + 64 * 64) + 2 * batch * (2 * 64 * 64 + 2 * 64 * 32)
    assert r["tensor"]["algorithmic_flops_per_launch"] == flops
    assert r["tensor"]["peak"] == 1500.0  # the sustained bf16 figure for a kernel inside a long step
    sr = r["issued_16B_accesses"]
    assert sr["reductions_per_launch"] == batch * 16 * 6
    assert sr["frac"] == pytest.approx(sr["achieved_per_s"] / 2e11)


def test_encode_roofline_is_the_l2_gather(bench):
    batch = 1 << 18
    r = bench.roofline_of("encode", {"encode": 0.07}, "fp16", PK, "measured", batch, 1, 0, D, 16, 2, L2PK)
    assert r["bound"] == "l2"
    assert r["algorithmic_bytes_per_launch"] == batch * (8 * 16 * 2 * 2 + 8 * 4)
    assert r["peak"] == pytest.approx(3e11 * 16 / 1e9)
    assert r["hbm"]["algorithmic_bytes_per_launch"] == batch * (8 * 16 * 2 * 2 + 2 * 32 + 8 * 4 + 4)
    assert r["issued_16B_accesses"]["loads_per_launch"] == batch * (16 * 5 + 8)


def test_traffic_is_withheld_when_the_sources_changed(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic_cfg2.txt").write_text("# csrc_sha256 0000\nk_adam 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_digest", lambda: "0000")
    assert bench.ncu_traffic("k_adam")[0] == 123
    monkeypatch.setattr(bench, "csrc_digest", lambda: "1111")
    val, note = bench.ncu_traffic("k_adam")
    assert val is None and "changed" in note


def test_fp32_mlp_is_an_alu_roofline(bench):
    r = bench.roofline_of("mlp", {"mlp": 2.0}, "fp32", PK, "measured", 1 << 18, 1, 0, D, 16, 2, L2PK)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2000.0 * 1e6 / 1e12)


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--cpu-points", "2048"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_render_gather_roofline_counts_corner_bytes_and_issue_rate(bench):
    ns, ms = 100_000_000, 8.0
    l2 = {"l1_gather_loads_per_s": 7e11, "gather_loads_per_s": 3e11}
    r = bench.gather_roofline(ns, ms, 16, 2, 32, PK, "measured", l2)
    assert r["algorithmic_bytes_per_frame"] == ns * 8 * 16 * 2 * 2  # 8 corners x L levels x F x 2 B
    assert r["frac"] == pytest.approx(r["achieved"] / (7e11 * 16 / 1e9))
    assert r["issued_corner_loads"]["per_frame"] == ns * 16 * 8
    assert r["hbm"]["bytes_per_sample"] == 12 + 2 * 32
    iss = r["issue"]  # warp instructions against one per SM sub-partition and cycle
    ipl = bench.RENDER_GATHER_INSTR_PER_SAMPLE_LEVEL
    assert iss["achieved_per_s"] == pytest.approx(ipl * ns * 16 / 32 / (ms / 1e3))
    assert iss["frac"] == pytest.approx(iss["achieved_per_s"] / iss["peak_per_s"])
    assert iss["peak_per_s"] % (4 * 2000e6) == 0  # 4 per SM per cycle at the maximum clock
