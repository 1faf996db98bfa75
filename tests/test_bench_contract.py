"""The benchmark's JSON contract on the paths that run without a GPU: the
CPU reference arm (the oracle timed on the host cores) and its refusal on
workloads it does not time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + list(args),
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _bench("--impl", "reference", "--workload", "gapped_n256_fp64", "--steps", "2", "--warmup", "3")
    assert d["impl"] == "reference"
    assert d["metric"] == "fermi_expansion_solves_per_s" and d["unit"] == "solves/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "gapped_n256_fp64" and d["config"]["n"] == 256
    assert d["config"]["parallelism"] == "single"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_default_workload_is_sampled():
    """The default workload (n = 16384, finite T) is timed on a bounded
    sample: the oracle's density of the same recipe at n = 1024, scaled by
    n^3 to the full size and labelled so."""
    d = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and "unavailable" not in d
    assert d["config"]["workload"] == "fermi_n16384" and d["config"]["n"] == 16384
    assert d["config"]["kT"] == 0.003
    assert d["value"] > 0 and "n=1024" in d["cpu_baseline"]["sample"] and "^3" in d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"]


def test_reference_arm_unavailable_on_many_problem_workloads():
    d = _bench("--impl", "reference", "--workload", "ragged_batch64")
    assert d["impl"] == "reference" and "unavailable" in d


def test_traffic_records_match_the_kernel_sources():
    """Every DRAM-traffic record in profiles/traffic.json was taken on the
    kernel source as it stands (its sha256 matches), so the bench line's
    roofline carries the measured traffic, not null; a kernel edit without a
    new capture fails here instead of silently dropping the figure."""
    sys.path.insert(0, ROOT)
    import bench
    tab = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    src = {"k_sym_mma": "k_mma.cu", "k_digit_mma": "k_digit.cu", "k_fp64_step": "k_fp64.cu"}
    assert tab
    for key in tab:
        kernel, workload = key.split("@")
        got = bench.traffic_record(kernel, src[kernel], workload)
        assert got is not None and got > 0, key
