"""The bench's reference arm (the CPU oracle, runnable here) prints one JSON
line with every key of the bench contract, the same config keys as the GPU
arm's line, and a cpu_baseline describing its own run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CONTRACT = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline", "impl"}
CONFIG = {"workload", "n", "nnz", "m", "bloom_bits", "bloom_b", "khash_k", "onehash_k", "per_edge_jaccard",
          "passes"}


def test_reference_line_keys():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "er4096", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert CONTRACT <= set(line), CONTRACT - set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert CONFIG <= set(line["config"]), CONFIG - set(line["config"])
    assert line["config"]["workload"] == "er4096" and line["config"]["passes"] == ["bloom", "khash"]
    assert line["config"]["m"] * 2 == line["config"]["nnz"]  # symmetric, no self-loops
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["value"] > 0 and line["higher_is_better"] is True
