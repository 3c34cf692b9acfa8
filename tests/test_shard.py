"""The vertex-partitioned run (paper_2208_11469_gb300/shard.py, Sec. VIII-F)
on CPU ranks: two and three gloo processes run the driver with the oracle
doing each rank's compute (sketch rows of its own vertices, per-edge counts
and estimates of its own upper edges). The driver's partition, sketch-row
exchange and reductions must give the single-process oracle's results: the
integer histogram bit for bit, the triangle total and every T_v within 1e-9
relative, LCC within 1e-5."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RTOL_F64 = 1e-9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """The four per-rank calls of shard.run on the CPU oracle. Sketch rows
    travel as bytes: Bloom filters packed 64 bits per word, MinHash rows as
    the oracle's int32 element ids."""

    def __init__(self, rp, cl, est, *, l=0, b=0, k=0, seed=1):
        from oracle import oracle as O
        self.O, self.rp, self.cl, self.est = O, rp, cl, est
        self.l, self.b, self.k, self.seed = l, b, k, seed
        self.kind = {O.EST_BF_AND: "bloom", O.EST_BF_L: "bloom", O.EST_KH: "khash", O.EST_1H: "onehash"}[est]
        self.eu, self.ev = O.upper_edges(rp, cl)
        self.table = None

    def _sub(self, a, b):
        rp = self.rp[a:b + 1] - self.rp[a]
        return rp.astype(np.int32), self.cl[self.rp[a]:self.rp[b]].astype(np.int32)

    def build_rows(self, a, b):
        O = self.O
        rp, cl = self._sub(a, b)
        if self.kind == "bloom":
            words = self.l // 64
            rows = O.bloom_pack(O.bloom_bits(rp, cl, self.l, self.b, self.seed), words).view(np.uint8)
        elif self.kind == "khash":
            rows = O.khash(rp, cl, self.k, self.seed).view(np.uint8)
        else:
            rows = O.onehash(rp, cl, self.k, self.seed).view(np.uint8)
        return torch.from_numpy(np.ascontiguousarray(rows).reshape(b - a, -1))

    def set_table(self, table):
        t = table.numpy()
        if self.kind == "bloom":
            words = t.view(np.uint64).reshape(t.shape[0], -1)
            bits = np.unpackbits(words.view(np.uint8), axis=1, bitorder="little")[:, : self.l]
            self.table = np.ascontiguousarray(bits, dtype=np.uint8)
        else:
            self.table = np.ascontiguousarray(t.view(np.int32).reshape(t.shape[0], -1))

    def partial(self, a, b):
        O = self.O
        sel = (self.eu >= a) & (self.eu < b)
        pu, pv = self.eu[sel], self.ev[sel]
        cnt = O.pair_counts(self.rp, self.cl, self.est, self.table, pu, pv, seed=self.seed)
        e = O.pair_estimates(self.rp, self.est, cnt, pu, pv, l=self.l, b=self.b, k=self.k)
        n = self.rp.size - 1
        sums = np.zeros(n)
        np.add.at(sums, pu, e)
        np.add.at(sums, pv, e)
        return torch.from_numpy(sums), torch.from_numpy(self._hist(cnt, pu, pv))

    def _hist(self, cnt, pu, pv):
        d = self.O.degrees(self.rp).astype(np.int64)
        c = np.asarray(cnt["count"], np.int64)
        ds = d[pu] + d[pv]
        if self.kind == "bloom":
            return np.bincount(c, minlength=self.l + 1).astype(np.int64)
        hk = self.k + 1
        key = c if self.kind == "khash" else np.asarray(cnt["K"], np.int64) * hk + c
        bins = hk if self.kind == "khash" else hk * hk
        return np.concatenate([np.bincount(key, minlength=bins), np.bincount(key, weights=ds, minlength=bins)
                               .astype(np.int64)])

    def finalize(self, hist, sums):
        O = self.O
        h = hist.numpy()
        if self.kind == "bloom":
            j = np.arange(self.l + 1)
            f = O.est_and(j, self.l, self.b) if self.est == O.EST_BF_AND else O.est_limit(j, self.b)
            tc = float(np.dot(h.astype(np.float64), f)) / 3.0
        else:
            hk = self.k + 1
            bins = h.size // 2
            i = np.arange(bins)
            K = np.full(bins, self.k) if self.kind == "khash" else i // hk
            c = i % hk
            r = np.where(K + c > 0, c / np.maximum(K + c, 1), 0.0)
            tc = float(np.dot(h[bins:].astype(np.float64), r)) / 3.0
        s = sums.numpy()
        d = O.degrees(self.rp).astype(np.float64)
        T = s / 2.0
        with np.errstate(divide="ignore", invalid="ignore"):
            lcc = np.where(d >= 2, 2.0 * T / np.where(d >= 2, d * (d - 1.0), 1.0), 0.0)
        return {"tc": tc, "tri": T, "lcc": lcc, "hist": h}


CASES = {
    "bloom": dict(est=1, l=256, b=2),
    "khash": dict(est=3, k=16),
    "onehash": dict(est=4, k=8),
}


def _graph():
    from paper_2208_11469_gb300 import synth
    rp, cl = synth.rmat(11, 8, seed=5)
    return rp.numpy().astype(np.int32), cl.numpy().astype(np.int32)


def _worker(rank, world, port, out_dir, case):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2208_11469_gb300 import shard
    rp, cl = _graph()
    kw = dict(CASES[case])
    est = kw.pop("est")
    ops = OracleOps(rp, cl, est, **kw)
    out = shard.run(ops, np.diff(rp), rank, world)
    with open(os.path.join(out_dir, f"{case}_{rank}.json"), "w") as f:
        json.dump({"tc": out["tc"], "tri": out["tri"].tolist(), "lcc": out["lcc"].tolist(),
                   "hist": out["hist"].tolist(), "range": list(out["range"])}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", ["bloom", "khash", "onehash"])
def test_sharded_run_equals_single_process_oracle(tmp_path, world, case):
    from oracle import oracle as O
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path), case), nprocs=world, join=True,
                       start_method="spawn")
    rp, cl = _graph()
    kw = dict(CASES[case])
    est = kw.pop("est")
    ref = O.analyze(rp, cl, est, seed=1, **kw)
    ops = OracleOps(rp, cl, est, **kw)
    want_hist = ops._hist(ref["counts"], ref["eu"], ref["ev"])
    got = [json.load(open(tmp_path / f"{case}_{r}.json")) for r in range(world)]
    ranges = [tuple(g["range"]) for g in got]
    assert ranges[0][0] == 0 and ranges[-1][1] == rp.size - 1
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    for g in got:
        assert np.array_equal(np.asarray(g["hist"], np.int64), want_hist)
        assert g["tc"] == pytest.approx(ref["tc"], rel=RTOL_F64)
        np.testing.assert_allclose(g["tri"], ref["T"], rtol=RTOL_F64, atol=1e-12)
        np.testing.assert_allclose(g["lcc"], ref["lcc"], rtol=1e-5, atol=1e-9)


def test_partition_balances_degree_plus_one():
    from paper_2208_11469_gb300 import shard
    rng = np.random.default_rng(3)
    d = rng.zipf(2.0, size=5000).clip(max=4000)
    for world in (1, 2, 3, 7, 16):
        b = shard.partition(d, world)
        assert b[0] == 0 and b[-1] == d.size and np.all(np.diff(b) >= 0)
        w = np.array([(d[b[r]:b[r + 1]] + 1).sum() for r in range(world)])
        # each range's work is within one vertex of the even share
        assert np.all(np.abs(w - (d + 1).sum() / world) <= d.max() + 1), (world, w)
    assert np.array_equal(shard.partition(np.zeros(0, np.int64), 3), np.zeros(4, np.int64))
