"""Timing of the CPU oracle on one chunk of a sampled workload.

TEST INFRASTRUCTURE (the CPU-baseline leg of bench.py): it runs the oracle
as it stands — the builders of Sec. II-D, the per-pair counts and estimators
of Sec. IV and the per-edge reductions of Sec. VII — on a chunk of rows of a
large graph and reports how long each phase took. It imports neither torch
nor the CUDA library, so bench.py can run one copy per host core as plain
subprocesses:

    python -m oracle.sample_timing CHUNK.npz RESULT.json

CHUNK.npz holds a sub-CSR (rp int32 [R+1], cl int32 [nnz_R] with the graph's
own neighbour ids, so every sketch row equals the whole graph's), the number
of pairs to intersect, the pass table's row count, two seeds and a JSON list
of passes: {"name", "est", "l", "b", "k"}.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from oracle import oracle as O

_KIND = {O.EST_BF_AND: "bloom", O.EST_BF_L: "bloom", O.EST_BF_OR: "bloom", O.EST_BF_SS: "bloom",
         O.EST_KH: "khash", O.EST_1H: "onehash", O.EST_1H_LITERAL: "onehash", O.EST_1H_KMV: "onehash"}


def sketch_key(p: dict):
    kind = _KIND[p["est"]]
    return (kind, p["l"], p["b"]) if kind == "bloom" else (kind, p["k"])


def time_chunk(rp, cl, passes, pairs: int, table_rows: int = 0, seed: int = 1, pair_seed: int = 0) -> dict:
    """Build every distinct sketch of `passes` over the chunk's rows (timed),
    then run each pass over `pairs` pairs (timed): integer counts, double
    estimates, their sum (the TC total) and the per-vertex sums at both ends
    (np.add.at, as oracle.analyze does). Returns the seconds of each phase.

    The pass reads a table of max(R, table_rows) rows, each a copy of one of
    the chunk's R sketch rows (every row at least once), so that its memory
    footprint is that of a whole-graph pass rather than of the small chunk;
    pair endpoints are drawn over the table with probability proportional
    to the degree of the copied row, as the endpoints of a uniformly drawn
    edge are. The table and the pairs are set up untimed."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    cl = np.ascontiguousarray(cl, dtype=np.int32)
    R = rp.size - 1
    O.lib()  # load before timing
    sk, t_build = {}, {}
    for p in passes:
        key = sketch_key(p)
        if key in sk:
            continue
        t0 = time.perf_counter()
        if key[0] == "bloom":
            sk[key] = O.bloom_bits(rp, cl, key[1], key[2], seed)
        elif key[0] == "khash":
            sk[key] = O.khash(rp, cl, key[1], seed)
        else:
            sk[key] = O.onehash(rp, cl, key[1], seed)
        t_build["_".join(map(str, key))] = time.perf_counter() - t0
    # pass tables and pairs (untimed)
    rng = np.random.default_rng(pair_seed)
    T = max(R, int(table_rows))
    src = np.concatenate([np.arange(R), rng.integers(0, R, size=T - R)]) if R else np.zeros(0, np.int64)
    rng.shuffle(src)
    tab = {key: np.ascontiguousarray(a[src]) for key, a in sk.items()}
    d = np.diff(rp).astype(np.int64)[src]
    trp = np.zeros(T + 1, dtype=np.int64)
    trp[1:] = np.cumsum(d)
    trp = trp.astype(np.int32)  # row offsets carrying each table row's degree
    if d.sum() > 0:
        w = d / d.sum()
        pu = rng.choice(T, size=pairs, p=w).astype(np.int32)
        pv = rng.choice(T, size=pairs, p=w).astype(np.int32)
    else:
        pu = pv = np.zeros(pairs, np.int32)
    t_pass, total = {}, 0.0
    for p in passes:
        t0 = time.perf_counter()
        cnt = O.pair_counts(trp, cl, p["est"], tab[sketch_key(p)], pu, pv, seed=seed)
        e = O.pair_estimates(trp, p["est"], cnt, pu, pv, l=p["l"], b=p["b"], k=p["k"])
        S = np.zeros(T, dtype=np.float64)
        np.add.at(S, pu, e)
        np.add.at(S, pv, e)
        total += float(e.sum())
        t_pass[p["name"]] = time.perf_counter() - t0
    return {"rows": int(R), "entries": int(cl.size), "pairs": int(pairs), "table_rows": int(T),
            "t_build": t_build, "t_pass": t_pass, "build_s": float(sum(t_build.values())),
            "pass_s": float(sum(t_pass.values())), "checksum": total}


def main(argv):
    src, dst = argv[1], argv[2]
    z = np.load(src)
    passes = json.loads(str(z["passes"]))
    out = time_chunk(z["rp"], z["cl"], passes, int(z["pairs"]), int(z["table_rows"]), seed=int(z["seed"]),
                     pair_seed=int(z["pair_seed"]))
    with open(dst, "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main(sys.argv)
