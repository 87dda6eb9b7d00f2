"""CPU check of bench.py's reference arm (the oracle timed on host cores):
it runs without a GPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    # the line names what it timed: the oracle's FP64 sample, one RHS
    assert d["config"]["nrhs"] == 1 and d["config"]["precision"] == "fp64" and d["config"]["n"] == 8
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["host_cores"] >= 1


def test_traffic_record_is_tied_to_source_and_workload():
    """roofline.traffic comes from profiles/traffic.json only for the workload
    and the executor source it was captured on."""
    sys.path.insert(0, ROOT)
    import importlib
    bench = importlib.import_module("bench")
    f = bench._factor_traffic(24, 1e-4, "fp32")
    a = bench._factor_traffic(24, 1e-4, "fp32", "exec_kernel_apply", 8)
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    same_src = rec["exec_kernel_factor"]["exec_cu_blob"] == bench._blob_sha1(
        os.path.join(ROOT, "paper_2211_11303_gb300", "csrc", "exec.cu"))
    if same_src:
        assert f == rec["exec_kernel_factor"]["dram_bytes_per_launch"] > 0
        assert a == rec["exec_kernel_apply"]["dram_bytes_per_launch"] > 0
    else:
        assert f is None and a is None
    assert bench._factor_traffic(16, 1e-4, "fp32") is None
    assert bench._factor_traffic(24, 1e-6, "fp32") is None
    assert bench._factor_traffic(24, 1e-4, "fp64") is None
    assert bench._factor_traffic(24, 1e-4, "fp32", "exec_kernel_apply", 4) is None
