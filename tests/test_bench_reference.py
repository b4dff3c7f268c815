"""bench.py --impl reference (the CPU oracle arm) on the small classic workload:
one JSON line with the contract's keys, no GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "cfg1",
                        "--steps", "2", "--warmup", "3", "--ref-queries-per-step", "5"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "k-mers/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_bench_rejects_short_warmup():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "2"], capture_output=True,
                       text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_traffic_record_matches_the_gather_sources():
    # the committed ncu record (roofline.traffic) was taken on the gather
    # kernel as it is now: its source hash matches, and it states the slice width
    # and the physical DRAM bytes of one launch
    sys.path.insert(0, ROOT)
    import bench
    csrc = os.path.join(ROOT, "paper_1905_09624_gb300", "csrc")
    rec = bench.traffic_record([os.path.join(csrc, "gather.cu"), os.path.join(csrc, "gather_common.cuh")])
    assert rec is not None, "gather sources changed since profiles/gather_batched_cfg2_dram.txt was captured"
    assert rec["slice_bytes"] in (128, 256)
    assert 0.6e9 < rec["dram_bytes"] < 12.26e9  # at least the index once, at most the logical row bytes


def test_config_traffic_records_match_their_sources():
    # the records behind the configs object's physical row GB/s (cfg3: one
    # step's four class launches; cfg4: one launch) match the current kernels
    # and hold between the index once and the logical row bytes
    sys.path.insert(0, ROOT)
    import bench
    csrc = os.path.join(ROOT, "paper_1905_09624_gb300", "csrc")
    bounds = {"cfg3": (8.0e9, 3.77e12), "cfg4": (0.47e9, 5.03e11)}
    for name, (record, srcs) in bench.CONFIG_RECORDS.items():
        rec = bench.traffic_record([os.path.join(csrc, f) for f in srcs], record)
        assert rec is not None, f"{name}: kernel sources changed since profiles/{record} was captured"
        lo, hi = bounds[name]
        assert lo < rec["dram_bytes"] < hi, (name, rec)

