"""Host logic of bench.py on CPU: the clock-sample summary (median SM clock, throttle
reasons) and the ncu counter record of the force kernel, which is used only while the
kernel source it was taken on is unchanged."""
import hashlib
import json
import os

import pytest


@pytest.fixture()
def bench():
    import bench as b

    return b


def test_clock_summary_median_and_reasons(bench, tmp_path):
    c = bench.ClockSampler(tmpdir=str(tmp_path))
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbage line"]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    assert not os.path.exists(c.path)  # the temporary file is removed once read


def test_clock_summary_without_samples(bench, tmp_path):
    c = bench.ClockSampler(tmpdir=str(tmp_path))
    assert c.summary() is None


def _fake_tree(root, src_text, rec):
    (root / "profiles").mkdir()
    csrc = root / "paper_1105_5613_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_force.cu").write_text(src_text)
    (root / "profiles" / "force_traffic.json").write_text(json.dumps(rec))


def test_force_counters_follow_the_source(bench, tmp_path, monkeypatch):
    src = "// kernel source\n"
    rec = {"block_z": 4, "bytes_per_particle": 284.0, "warp_inst_per_particle": 150.0,
           "k_force_cu_sha1": hashlib.sha1(src.encode()).hexdigest()}
    _fake_tree(tmp_path, src, rec)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.force_traffic(1000) == pytest.approx(284000.0)
    issue = bench.force_issue(1_000_000, 1.0, 4, 2000.0, 152)
    # 150e6 warp instructions in 1 ms against 152 SMs x 4 per cycle at 2 GHz
    assert issue["frac"] == pytest.approx(1.5e11 / (152 * 4 * 2e9))
    assert bench.force_issue(1_000_000, 1.0, 8, 2000.0, 152) is None  # another block shape
    # a record without a skin is of the skin 0.3; another skin has other lists
    assert bench.force_traffic(1000, 0.3) == pytest.approx(284000.0)
    assert bench.force_traffic(1000, 0.4) is None
    assert bench.force_issue(1_000_000, 1.0, 4, 2000.0, 152, 0.4) is None
    # any change of the source voids the record
    (tmp_path / "paper_1105_5613_gb300" / "csrc" / "k_force.cu").write_text(src + " ")
    assert bench.force_traffic(1000) is None
    assert bench.force_issue(1_000_000, 1.0, 4, 2000.0, 152) is None


def test_a_failing_secondary_leg_is_reported_not_fatal(bench):
    def boom(x):
        raise MemoryError(f"no room for {x} particles")

    assert bench.optional_leg(lambda a, b: a + b, 2, 3) == 5
    r = bench.optional_leg(boom, 1024191500)
    assert r == {"error": "MemoryError: no room for 1024191500 particles"}


def test_bench_runs_end_to_end_against_standins():
    """Every leg of bench.py through its host code, with the library and CUDA replaced by
    stand-ins (tests/bench_standins.py); the one JSON line carries every key of the
    contract and no leg reports an error."""
    import subprocess
    import sys

    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "bench_standins.py")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "roofline", "cpu_baseline", "gpu_launches"):
        assert k in d, k
    assert d["gpu_launches"] == 3 * 16 + 2
    for leg in ("fp64", "soft_sphere", "replicas", "large", "cpu_baseline", "fma_probe"):
        assert "error" not in d[leg], d[leg]
    assert d["roofline"]["peak"] == d["fma_probe"]["fp32_tflops"]
    assert {"roofline", "phases_ms_per_step", "rebuilds_per_step"} <= set(d["large"]["mixed"])
    assert {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"} <= set(d["e2e"])
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(d["roofline"])
    assert {"value", "unit", "cores", "kind", "sample"} <= set(d["cpu_baseline"])


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` (the oracle, on the host) prints one JSON line with the
    same metric and config as the library's arm, marked as the reference."""
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] >= 3
    assert d["metric"].startswith("particle-steps/s") and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the config names the bounded sample this arm times, and what it is a sample of
    assert d["config"]["n_particles"] == 4 * 20 ** 3
    assert "N=32000" in d["config"]["workload"] and "sample_of" in d["config"]
