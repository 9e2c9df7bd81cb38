"""The reference arm of bench.py (the CPU oracle) prints one JSON line with the
contract's keys; it needs no GPU, so it runs here at a small size."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "48",
                          "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "steps/s" and d["higher_is_better"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert "workload" in d["config"]



def test_reference_arm_rank0_only():
    """With the environment a torchrun launch gives each rank (N = 2): rank 0 alone
    runs the oracle and prints the line, rank 1 exits 0 without work or output."""
    outs = {}
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT="29500")
        outs[rank] = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                     "--gpus", "2", "--n", "32", "--steps", "1", "--warmup", "3"],
                                    cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    for rank, out in outs.items():
        assert out.returncode == 0, (rank, out.stderr[-2000:])
    lines0 = [ln for ln in outs[0].stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines0) == 1
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert outs[1].stdout.strip() == ""
