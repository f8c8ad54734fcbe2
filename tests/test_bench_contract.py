"""bench.py's contract on the CPU: the reference arm (the FP64 oracle timed on the host cores) prints one
JSON line with the keys of the benchmark contract, and the ncu counter tables parse."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--envs", "4"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mrays/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["ray_tri_tests_per_s"] > 0 and d["cpu_baseline"]["full_step_s_extrapolated"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["metric"].startswith("Mrays/s at 1024 envs x 270x480")


def test_counter_tables_parse():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert len(b.kernel_source_hash()) == 16
    rows = current = 0
    for name in os.listdir(b.PROFILE_DIR):
        if name.startswith("k_trace_") and name.endswith("_traffic.md"):
            for line in open(os.path.join(b.PROFILE_DIR, name)):
                cells = [c.strip() for c in line.strip().strip("|").split("|")]
                if len(cells) == 7 and ":" in cells[0] and cells[1].startswith("k_trace<"):
                    assert int(cells[3]) + int(cells[4]) == int(cells[5]) and int(cells[6]) > 0
                    rows += 1
                    current += cells[2] == b.kernel_source_hash()
    assert rows >= 2
    # the committed counters were taken on the current kernel and builder sources (else the bench reports
    # traffic as null): recapture them after changing either
    assert current >= 2


def test_clock_samples_summary():
    """The clock record of the timed region: median SM clock, max clock and every active throttle reason."""
    import importlib.util
    import tempfile
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Active"]
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    c = b.ClockSampler(0)
    c.path = path
    out = c.summary()
    assert out == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert not os.path.exists(path)
    c2 = b.ClockSampler(0)
    c2.path = os.path.join(tempfile.gettempdir(), "does-not-exist.csv")
    assert c2.summary()["reasons"] == ["unsampled"]


def test_clock_rejection_rule():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod3", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not b.clocks_rejected(ok)
    assert not b.clocks_rejected(dict(ok, reasons=["sw_power_cap"], sm_mhz=1700.0))  # power cap: kept
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert b.clocks_rejected(dict(ok, reasons=[r]))
    assert b.clocks_rejected(dict(ok, sm_mhz=1400.0))          # well below max with no reason: a lock
    assert not b.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]})


def test_rooflines_follow_from_their_inputs():
    """The lead roofline is the issue one (bound alu) when counters exist, with the DRAM fraction beside it;
    the algorithmic-bytes block is labelled as such; every fraction is its achieved value over its peak."""
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert abs(b.issue_peak_g(152, 2070.0) - 1258.56) < 1e-9
    lead, algo = b.rooflines((1.2e9, 1.19e10), 12.4, 1790.0, 132710400, 6789.6, "measured", 152, 2070.0, 7.67,
                             3.89, 208)
    assert lead["bound"] == "alu" and lead["unit"] == "G warp instructions/s"
    assert abs(lead["achieved"] - 1.19e10 / 12.4e-3 / 1e9) < 1e-6
    assert abs(lead["frac"] - lead["achieved"] / lead["peak"]) < 1e-12 and lead["peak"] == b.issue_peak_g(152, 2070.0)
    assert abs(lead["dram_gbs"] - 1.2e9 / 12.4e-3 / 1e9) < 1e-6 and abs(lead["dram_frac"] - lead["dram_gbs"] / 6789.6) < 1e-12
    assert lead["traffic"] == 1.2e9 and lead["algorithmic"] is algo
    assert algo["bound"] == "hbm" and "L1/L2" in algo["achieved_is"]
    assert abs(algo["achieved"] - 1790.0 * 132710400 / 12.4e-3 / 1e9) < 1e-6
    assert abs(algo["frac"] - algo["achieved"] / 6789.6) < 1e-12
    lead2, algo2 = b.rooflines(None, 12.4, 1790.0, 132710400, 6789.6, "measured", 152, 2070.0, 7.67, 3.89, 208)
    assert algo2 is None and lead2["bound"] == "hbm" and lead2["traffic"] is None
