"""The bench's reference arm (the CPU oracle, runnable here) prints one JSON
line with every key of the bench contract, the same config keys as the GPU
arm's line, and a cpu_baseline describing its own run."""
import json
import os
import subprocess
import sys

import pytest

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


def test_thm71_radius():
    """Thm. 7.1's 95% deviation radius as the bench reports it: MinHash from the
    degree sums (the smaller of the two Hoeffding forms, each of which gives
    exactly delta back), Bloom AND only under the theorem's condition."""
    import math
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2208_11469_gb300 import synth
    rp, cl = synth.erdos_renyi(4096, 16.0, seed=1)
    d = np.diff(rp.numpy()).astype(np.float64)
    k, delta = 32, 0.05
    out = bench.tc_deviation_bounds(rp, [("kh", "minhash", 0, 0, k), ("bf", "bloom_and", 1024, 1, 0),
                                         ("bf_small", "bloom_and", 64, 16, 0), ("x", None, 0, 0, 0)], delta)
    t = out["kh"]["t"]
    p1 = 2 * math.exp(-18 * k * t * t / (np.sum(d * d) ** 2))
    p2 = 2 * math.exp(-9 * k * t * t / (4 * (d.max() + 1) * np.sum(d ** 3)))
    assert min(p1, p2) <= delta * (1 + 1e-9) and max(p1, p2) >= delta * (1 - 1e-9)
    m = d.sum() / 2
    b, l, dm = 1, 1024, d.max()
    C = math.exp(dm * b / (l - 1)) * l / b**2 - l / b**2 - dm / b
    tb = out["bf"]["t"]
    assert 2 * m * m * C / (9 * tb * tb) == pytest.approx(delta, rel=1e-12)
    assert out["bf_small"]["t"] is None and "0.499" in out["bf_small"]["reason"]  # 16 * max d > 0.499 * 64 ln 64
    assert out["x"] is None


def test_oracle_leg_samples_the_whole_graph():
    """The CPU leg's sample: uniformly drawn rows without repeats within a run
    of chunks, sub-CSRs that hold each sampled row's own neighbours (so their
    sketches are the whole graph's), pass tables no smaller than the rows, and
    a whole-graph time that scales the sample's phases by n/R and m/E."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import sample_timing as ST
    from paper_2208_11469_gb300 import synth
    rp, cl = synth.rmat(12, 8, seed=2)
    leg = bench.OracleLeg(rp, cl, dict(bench.WORKLOADS["er4096"]), 256, seed=3)
    chunks = leg.chunks(1200, 4000, 4)
    assert len(chunks) == 4 and all(c["pairs"] == 1000 for c in chunks)
    rpn, cln = rp.numpy(), cl.numpy()
    all_rows = np.concatenate([c["rows"] for c in chunks])
    assert all_rows.size == 1200 and np.unique(all_rows).size == 1200
    for c in chunks:
        d = np.diff(c["rp"])
        assert c["rp"][0] == 0 and d.sum() == c["cl"].size and c["table_rows"] >= d.size
        for i, v in enumerate(c["rows"]):
            assert np.array_equal(c["cl"][c["rp"][i]:c["rp"][i + 1]], cln[rpn[v]:rpn[v + 1]])
    r = ST.time_chunk(chunks[0]["rp"], chunks[0]["cl"], leg.passes, 500, 2000, pair_seed=1)
    assert r["pairs"] == 500 and r["table_rows"] == 2000 and r["rows"] == chunks[0]["rp"].size - 1
    assert set(r["t_pass"]) == {"bloom", "khash"} and r["build_s"] > 0 and r["pass_s"] > 0
    rate, T = leg._rate(2.0, 1.0, 100, 1000)
    assert T == pytest.approx(2.0 * leg.n / 100 + 1.0 * leg.m / 1000)
    assert rate == pytest.approx(2 * leg.m / T)


def test_source_fingerprint_ignores_comments_only():
    """The traffic gate's fingerprint follows the code of the pass sources:
    comments and whitespace do not move it, any code token does, and comment
    markers inside string or character literals are code."""
    import bench
    a = "int f(int x) { return x + 1; } // add one\n"
    b = "/* a comment */ int  f(int x)\n{ return x + 1; }\n"
    c = "int f(int x) { return x + 2; }\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
    s = 'const char *u = "http://x"; char q = \'/\';'
    assert bench.code_only(s) == s
    assert len(bench.source_fingerprint()) == 64
