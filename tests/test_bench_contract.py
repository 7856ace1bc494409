"""The benchmark's reference arm (the oracle on the host cores) prints one
JSON line with the keys the measurement contract names; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "softmax_n20k_d1000", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "softmax_n20k_d1000"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_record_needs_the_same_source_and_configuration():
    # the DRAM/algorithmic ratio of a capture applies only to the kernel source
    # and the configuration it was taken on
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kernel in ("gather", "gather_prefix", "k_dense"):
        cfg = dict(rec[kernel]["config"])
        got = bench._traffic_record(kernel, cfg)
        import hashlib
        src = os.path.join(ROOT, "paper_2311_02573_gb300", "csrc", rec[kernel]["source"])
        current = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec[kernel]["source_sha"]
        assert (got is not None) == current
        for key, other in (("rho", 0.9), ("dtype", "f32"), ("cutover", 4), ("N", 20_000)):
            assert bench._traffic_record(kernel, dict(cfg, **{key: other})) is None
