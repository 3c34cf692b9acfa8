"""Vertex-partitioned run of the sketched path over torch.distributed ranks.

The distributed form of ProbGraph (Sec. VIII-F): the vertices are split among
the processes, each process builds the sketches of its own vertices (a
sketch row depends on its own neighbourhood only), the sketch rows are
exchanged so that every process can read the rows its edges need, each
process estimates the upper edges (u, v) of its own vertices u, and the
integer count histograms and the per-vertex sums are added over the
processes. The paper sends whole sketches point to point; here the exchange
is one all-gather of the sketch table (the table is small beside the CSR:
0.94 GB of Bloom filters for a 4.16 GB CSR at the 25% budget), and the
reductions are two all-reduces. Every rank holds the whole CSR and its edge
index.

The per-rank compute goes through an `ops` object with four calls, so the
same driver runs the CUDA library (DeviceOps) on GPU ranks and any other
implementation of the same four calls elsewhere:
    build_rows(a, b)      -> uint8 [b - a, stride]: sketch rows of vertices a..b-1
    set_table(table)      -> take the exchanged uint8 [n, stride] sketch table
    partial(a, b)         -> (float64 [n] sums, int64 [bins] hist) of the upper
                             edges (u, v) with a <= u < b
    finalize(hist, sums)  -> dict(tc=..., lcc=..., tri=...)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch
import torch.distributed as dist


def partition(degrees, world: int) -> np.ndarray:
    """Contiguous vertex ranges [bounds[r], bounds[r+1]) with near-equal work:
    the builds cost per CSR entry and the pass per upper edge, both in
    proportion to the degree, plus a per-vertex part; a vertex weighs d_v + 1."""
    d = np.asarray(degrees, dtype=np.int64)
    n = d.size
    w = np.cumsum(d + 1)
    total = int(w[-1]) if n else 0
    bounds = np.zeros(world + 1, dtype=np.int64)
    for r in range(1, world):
        bounds[r] = int(np.searchsorted(w, total * r / world, side="left")) if n else 0
    bounds[world] = n
    return np.maximum.accumulate(bounds)


def all_gather_rows(local: torch.Tensor, bounds: np.ndarray, world: int, group=None) -> torch.Tensor:
    """The whole sketch table [n, stride] from every rank's rows
    [bounds[r+1] - bounds[r], stride] (rows padded to the largest range for
    the collective, then cut back)."""
    stride = local.shape[1]
    sizes = np.diff(bounds)
    mx = int(sizes.max()) if world else 0
    pad = torch.zeros((mx, stride), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: int(sizes[r])] for r in range(world)], dim=0)


def run(ops, degrees, rank: int, world: int, group=None) -> dict:
    """One vertex-partitioned run on this rank. Returns the finalized totals
    (identical on every rank) and this rank's range."""
    bounds = partition(degrees, world)
    a, b = int(bounds[rank]), int(bounds[rank + 1])
    local = ops.build_rows(a, b)
    ops.set_table(all_gather_rows(local, bounds, world, group))
    sums, hist = ops.partial(a, b)
    if world > 1:
        dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)  # int64: exact
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    out = ops.finalize(hist, sums)
    out["range"] = (a, b)
    out["bounds"] = bounds
    return out


class DeviceOps:
    """The four calls on the CUDA library (include/pg.h): row-range builds
    through a CSR view of rows a..b-1 (pg_build_bloom / pg_build_minhash),
    pg_partial_sums and pg_finalize_sums. g: pg.Graph with its index;
    kind/bits/b/k/seed: the sketch; est: the estimator."""

    def __init__(self, g, kind: int, est: int, *, bits: int = 0, b: int = 0, k: int = 0, seed: int = 1):
        from paper_2208_11469_gb300 import pg
        self.pg, self.g, self.est = pg, g, est
        self.kind, self.bits, self.b, self.k, self.seed = kind, bits, b, k, seed
        self.stride = pg.sketch_stride(kind, bits, k)
        self.ws_build = torch.empty(max(pg.build_workspace_bytes(g), 16), dtype=torch.uint8, device=g.device)
        self.sk = None

    def build_rows(self, a: int, b: int) -> torch.Tensor:
        pg, g = self.pg, self.g
        rows = torch.empty((max(b - a, 0), self.stride), dtype=torch.uint8, device=g.device)
        if b > a:
            view = pg.Csr(g.row_ptr.data_ptr() + 4 * a, g.col.data_ptr() if g.col.numel() else None, b - a, g.nnz)
            desc = pg.SketchDesc(self.kind, self.bits, self.b, self.k, self.seed & 0xFFFFFFFF, b - a, self.stride,
                                 rows.data_ptr())
            fn = pg.lib().pg_build_bloom if self.kind == pg.SK_BLOOM else pg.lib().pg_build_minhash
            pg._check(fn(ctypes.byref(view), ctypes.byref(desc), ctypes.c_void_p(self.ws_build.data_ptr()),
                         self.ws_build.numel(), pg._stream()), "row-range sketch build")
        return rows

    def set_table(self, table: torch.Tensor) -> None:
        pg = self.pg
        data = table.contiguous().view(-1)
        self.sk = pg.Sketch(self.kind, self.bits, self.b, self.k, self.seed, self.g.n, self.stride, data)

    def partial(self, a: int, b: int):
        return self.pg.partial_sums(self.g, self.sk, self.est, a, b)

    def finalize(self, hist: torch.Tensor, sums: torch.Tensor) -> dict:
        pg = self.pg
        tc, lcc, tri = pg.finalize_sums(self.g, self.sk, self.est, hist, sums)
        return {"tc": pg.read_tc_result(tc), "lcc": lcc, "tri": tri, "hist": hist}
