"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
the one JSON line the benchmark contract asks for, and the non-zero ranks of
a multi-rank launch exit without work."""

import hashlib
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "1", "--cpu-sample-cells", "3000", "--cpu-sample-rows", "100"],
                          capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_the_contract_line():
    p = _run()
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [l for l in p.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "cells/s"
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-3000:]
    assert p.stdout.strip() == ""


def test_roofline_traffic_only_for_the_source_it_was_measured_on(tmp_path, monkeypatch):
    # the committed per-launch DRAM bytes are reported while the kernel's
    # source is the one the counters were taken on, and dropped otherwise
    sys.path.insert(0, ROOT)
    import bench
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    rec = t["screen_tc_kernel"]
    src = open(os.path.join(ROOT, "paper_2407_19892_gb300", "csrc", "k_topk_tc.cu"), "rb").read()
    current = rec["source_sha1"] == hashlib.sha1(src).hexdigest()
    want = rec["dram_bytes_per_launch"] if current else None
    assert bench.kernel_traffic("k_topk_tc.cu", "screen_tc_kernel") == want
    assert bench.kernel_traffic("k_topk_tc.cu", "no_such_kernel") is None
    # a copy of the tree whose screen source differs by one byte: no traffic
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(t))
    csrc = tmp_path / "paper_2407_19892_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = open(os.path.join(ROOT, "paper_2407_19892_gb300", "csrc", "k_topk_tc.cu"), "rb").read()
    (csrc / "k_topk_tc.cu").write_bytes(src + b" ")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k_topk_tc.cu", "screen_tc_kernel") is None
    (csrc / "k_topk_tc.cu").write_bytes(src)
    src = open(os.path.join(ROOT, "paper_2407_19892_gb300", "csrc", "k_topk_tc.cu"), "rb").read()
    current = rec["source_sha1"] == hashlib.sha1(src).hexdigest()
    want = rec["dram_bytes_per_launch"] if current else None
    assert bench.kernel_traffic("k_topk_tc.cu", "screen_tc_kernel") == want


def test_clock_samples_give_median_max_and_throttle_reasons(tmp_path):
    # nvidia-smi's csv rows as the sampler receives them (one malformed line)
    sys.path.insert(0, ROOT)
    import bench

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    csv = tmp_path / "clocks.csv"
    csv.write_text("0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                   "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                   "garbage line\n"
                   "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = Done(), str(csv)
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not csv.exists()
