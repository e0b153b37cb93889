"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one JSON line with
the keys the measurement contract names (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--cpu-qp", "1", "--cpu-q", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "processes/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "morse-diamond-2atom-16x16x16-145q-adaptive-sigma"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["cpu_model"] and cb["nproc"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_one_core_oracle_sample_and_host_info():
    """The single-thread oracle figure the GPU arm adds to cpu_baseline (child process with
    OMP_NUM_THREADS=1) and the host description."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(cpu_qp=8, mesh=8, workload="allmodes")
    d = bench.cpu_oracle_one_core(args)
    assert d is not None and d["cores"] == 1 and d["value"] > 0 and "q' < 2" in d["sample"]
    model, n = bench.cpu_host_info()
    assert model and n >= 1


def test_default_steps_cover_the_sample_evenly():
    """The default step of the precision workload takes 29 of the 145 sampled q: the 5 batches
    partition the sample, so any multiple of 5 timed steps weights every q equally; the arms use
    its first 5 q."""
    sys.path.insert(0, ROOT)
    import bench
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = sys_argv
    assert a.q_per_step == 29 and a.w["n_sample"] == 145
    bl = bench.batches(a.w, a.q_per_step)
    assert len(bl) == 5 and all(len(b) == 29 for b in bl)
    allq = sorted(int(q) for b in bl for q in b)
    assert allq == sorted(int(q) for q in bench.q_sample(a.w)) and len(set(allq)) == 145
    assert bench.ARM_Q == 5
    assert a.w["name"] == "morse-diamond-2atom-16x16x16-145q-adaptive-sigma"
