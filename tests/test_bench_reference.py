"""The benchmark's reference arm (`bench.py --impl reference`): the FP64 oracle timed on the host
cores on a bounded sample of the headline workload, printed as one JSON line with the fields the
benchmark contract names (impl, metric, value, unit, the configuration, cpu_baseline and e2e).
Runs on the CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "1",
           "--ref-sample", "2048"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "geodesics/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 1
    assert d["metric"].startswith("face-crossings/sec and geodesics/sec")
    assert d["config"]["workload"].startswith("icosphere-s6-noisy") and d["config"]["global_batch"] == 2048
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "geodesics/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["crossings_per_s"] > 0


def test_traffic_record_matches_the_kernel_sources():
    """profiles/ncu_traffic.json holds the DRAM bytes and L2 requests of the walk and re-walk
    kernels as captured by ncu, keyed by the hash of their sources: the benchmark reports them
    only while the sources are those that were captured."""
    sys.path.insert(0, ROOT)
    import bench
    for k in ("k_walk_persistent", "k_bwd_rewalk"):
        assert bench.ncu_traffic(k) is not None, k
        assert bench.ncu_traffic(k, "lts_requests_per_launch") is not None, k
