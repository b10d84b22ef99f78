"""The benchmark's reference arm runs on the host: one JSON line with the
fields the ours-arm line carries (metric, value, unit, steps, config), the
reference marker, its CPU baseline description and an e2e entry."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "edge_evals/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "N=100 p=4" in d["config"]["workload"]


def test_traffic_capture_key_ignores_comments_only():
    """A DRAM traffic capture stays valid across a comment change and is
    voided by any change to the kernel code."""
    sys.path.insert(0, str(ROOT))
    import bench
    texts = [(ROOT / "paper_2106_15740_gb300" / "csrc" / f).read_text()
             for f in ("kernels.cu", "kernels.cuh", "qt_device.h")]
    base = bench.kernel_code_digest(texts)
    assert base == bench.kernel_code_digest()
    commented = [texts[0] + "\n// a remark\n/* another\n remark */\n", texts[1], texts[2]]
    assert bench.kernel_code_digest(commented) == base
    assert "constexpr int kFfCasLimit = 1 << 20;" in texts[1]
    changed = [texts[0], texts[1].replace("constexpr int kFfCasLimit = 1 << 20;", "constexpr int kFfCasLimit = 1 << 21;"),
               texts[2]]
    assert bench.kernel_code_digest(changed) != base
