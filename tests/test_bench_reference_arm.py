"""The benchmark's reference arm (the FP64 oracle timed on the host cores,
no GPU involved) prints one JSON line in the contract's shape; run on the CPU
with one step on the 64^3 sample grid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    # the oracle's configuration timings on a 16^3 grid here (64^3 by default)
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--oracle-configs-n", "16"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "DoF*cycles/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and "workload" in d["config"]
    c = d["oracle_configs"]
    assert c["threads"] == 1
    # the standalone 8^3 iteration and the PCG solves reach the tolerance
    assert c["standalone_8"]["relres"] <= 1e-8 and c["standalone_8"]["vcycles"] > 0
    assert [r["alpha"] for r in c["manufactured_pcg"]] == [0.01, 1.0, 100.0]
    assert all(r["relres"] <= 1e-8 and r["n"] == 16 for r in c["manufactured_pcg"])
    assert c["gradient"]["n"] == 16 and c["gradient"]["fwd_bwd_s"] > 0


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert res.returncode == 0 and res.stdout.strip() == ""
