"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on a
CPU and prints the one JSON line the benchmark contract asks for, naming the
same workload and metric as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--workload", "small", "--ref-patients", "16", "--ref-days", "2"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "simulated patient-years/s"
    assert d["unit"] == "patient-years/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["config"]["workload"].startswith("small: 1000 patients x 2016 periods")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "patient-years/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_clock_record_flags_throttling():
    """The clocks summary that decides whether a timed run stands: median SM
    clock under load, the maximum, and every throttle reason seen active in
    nvidia-smi's CSV (noheader, nounits) samples; unreadable lines are skipped."""
    import bench
    c = bench.Clocks(0)
    c.lines = [
        "0, 2070, 2070, 850.12, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1399.80, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A]",
        "0, [N/A], 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines.append("0, 1500, 2070, 700.0, 0x48, Not Active, Active, Not Active, Not Active")
    s = c.summary()
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and s["samples"] == 4
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]
