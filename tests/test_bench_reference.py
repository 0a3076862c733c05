"""The benchmark's CPU reference arm (the FP64 oracle on the host cores): one
JSON line with the contract's keys, finite throughput, the core count used."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "0"], capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-500:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("channel_3d_D3Q19_256x128x128")


def test_clock_sampler_parses_a_fake_nvidia_smi(tmp_path, monkeypatch):
    """The bench's clock record from an nvidia-smi stand-in on PATH: median SM
    clock, maximum, and the throttle reasons seen active."""
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!/bin/sh\n"
        "while true; do\n"
        "  echo '0, 2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
        "  echo '0, 1900, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
        "  sleep 0.02\n"
        "done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:" + os.environ.get("PATH", ""))
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r is not None and r["samples"] >= 2
    assert r["sm_max_mhz"] == 2070.0
    assert 1900.0 <= r["sm_mhz"] <= 2070.0
    assert r["reasons"] == ["sw_power_cap"]
