"""Host-side logic of the benchmark: the key that ties committed ncu counters
to the kernel source (comments do not change it, code does), the traffic
lookup that scales a capture by columns and refuses a stale one, and the
reference arm's JSON line (the oracle on the host cores; rank 0 only)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_key_ignores_comments_only():
    src = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    assert bench.source_key(src) == bench.source_key("// header\n" + src + "\n\n// trailing\n")
    assert bench.source_key(src) == bench.source_key(src.replace("// one more", "// a different remark"))
    assert bench.source_key(src) != bench.source_key(src.replace("x + 1", "x + 2"))
    assert bench.source_key(src) != bench.source_key(src.replace("return", "return  "))  # code text, not tokens


def test_kernel_source_has_no_comment_markers_inside_strings():
    """source_key cuts every line at its first //: that is only a comment
    cut while no string literal of the kernel file contains //."""
    text = open(os.path.join(ROOT, "paper_2212_05685_gb300", "csrc", "cheb_kernels.cu")).read()
    for line in text.splitlines():
        code = line.split("//", 1)[0]
        assert code.count('"') % 2 == 0, line
    assert "/*" not in text


def test_traffic_lookup_scales_and_refuses_stale_records():
    rec = json.load(open(os.path.join(ROOT, "profiles", "cheb_step_fp32_100x100.json")))
    key = rec["kernel_source_sha256_16"]
    got = bench.measured_traffic("cheb_step_fp32_100x100.json", key, 2 * rec["ldv"])
    assert got == 2 * rec["dram_bytes_per_launch"]
    assert bench.measured_traffic("cheb_step_fp32_100x100.json", "0" * 16, rec["ldv"]) is None
    assert bench.measured_traffic("no_such_profile.json", key, rec["ldv"]) is None
    # the benchmark reports the record only while the kernel source is the captured one
    current = bench.measured_traffic("cheb_step_fp32_100x100.json", bench.kernel_hash(), rec["ldv"])
    assert current == (rec["dram_bytes_per_launch"] if bench.kernel_hash() == key else None)


def _run_reference(env_extra):
    import subprocess
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--sample-cols", "1"], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=300)


def test_reference_arm_prints_the_contract_line():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the metric, the impl tag, its CPU-baseline record and a host-only e2e."""
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
