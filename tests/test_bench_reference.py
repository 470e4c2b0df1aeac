"""The reference arm of bench.py (the oracle on the host cores) follows the
native arm's configuration: its JSON line carries the same metric and the
contract's keys, and configurations it does not cover say so."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra) -> dict:
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *extra],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_reference_arm_small_configuration():
    sys.path.insert(0, ROOT)
    import bench
    line = _run("--config", "small", "--steps", "3", "--warmup", "3")
    assert line["impl"] == "reference" and line["metric"] == bench.SMALL_METRIC
    assert line["unit"] == "generations/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "generations/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "all 32 children" in line["cpu_baseline"]["sample"] or "32 of 32" in line["cpu_baseline"]["sample"]


def test_reference_arm_names_what_it_does_not_cover():
    line = _run("--config", "batching", "--steps", "3", "--warmup", "3")
    assert line["impl"] == "reference" and "batching" in line["unavailable"]
