"""Seeded synthetic graph inputs (Erdos-Renyi and R-MAT) as int32 CSR.

This module draws the random numbers that both the CUDA path and the CPU
oracle consume. It contains none of the method's arithmetic (no hashing, no
sketches, no estimators): it only turns seeds into simple undirected graphs.

The paper evaluates on SNAP/KONECT/DIMACS/WebGraph graphs and on Kronecker
graphs (Sec. VIII-A); none of those datasets are available here, so seeded
Erdos-Renyi G(n, p) and R-MAT graphs (the Kronecker family) stand in for them.

All graphs are returned as (row_ptr int32[n+1], col int32[nnz]) with every
undirected edge stored in both directions, sorted neighbour lists, no
self-loops and no duplicates (the CSR form of Sec. II-A).
"""
from __future__ import annotations

import numpy as np
import torch


def _rng(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def csr_from_pairs(u: torch.Tensor, v: torch.Tensor, n: int):
    """Symmetrise, drop self-loops and duplicates, sort; return int32 CSR.

    `u`, `v` are int64 tensors of equal length on any device."""
    keep = u != v
    u, v = u[keep], v[keep]
    a = torch.cat([u, v])
    b = torch.cat([v, u])
    del u, v
    key = torch.unique(a * n + b, sorted=True)
    del a, b
    src = torch.div(key, n, rounding_mode="floor")
    dst = (key - src * n).to(torch.int32)
    del key
    counts = torch.bincount(src, minlength=n)
    del src
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dst.device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    if int(row_ptr[-1]) >= 2**31:
        raise ValueError("graph has 2^31 or more CSR entries; int32 CSR cannot hold it")
    return row_ptr.to(torch.int32), dst


def erdos_renyi(n: int, avg_deg: float, seed: int, device="cpu"):
    """G(n, p) with p = avg_deg / (n - 1).

    The edge count M is drawn from Binomial(n(n-1)/2, p); given M, G(n, p)
    is uniform over graphs with M edges, so M distinct uniform pairs are
    drawn (duplicates rejected and redrawn)."""
    if n < 2:
        return torch.zeros(n + 1, dtype=torch.int32, device=device), torch.zeros(0, dtype=torch.int32, device=device)
    npairs = n * (n - 1) // 2
    p = min(1.0, avg_deg / (n - 1))
    M = int(np.random.Generator(np.random.PCG64(int(seed))).binomial(npairs, p))
    gd = _rng(seed + 0x5EED, device)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    while keys.numel() < M:
        need = M - keys.numel()
        draw = int(need * 1.1) + 16
        a = torch.randint(0, n, (draw,), generator=gd, device=device, dtype=torch.int64)
        b = torch.randint(0, n, (draw,), generator=gd, device=device, dtype=torch.int64)
        ok = a != b
        lo = torch.minimum(a, b)[ok]
        hi = torch.maximum(a, b)[ok]
        keys = torch.unique(torch.cat([keys, lo * n + hi]))
    if keys.numel() > M:
        perm = torch.randperm(keys.numel(), generator=gd, device=device)[:M]
        keys = keys[perm]
    u = torch.div(keys, n, rounding_mode="floor")
    v = keys - u * n
    return csr_from_pairs(u, v, n)


def rmat(scale: int, edgefactor: int, seed: int, a=0.57, b=0.19, c=0.19, d=0.05,
         permute: bool = True, device="cpu", n: int | None = None, samples: int | None = None):
    """R-MAT / Kronecker generator (the paper's Kronecker graphs, Sec. VIII-A).

    Draws edgefactor * 2^scale directed samples; at each of `scale` levels
    one uniform number picks a quadrant with probabilities (a, b, c, d).
    With `permute`, vertex labels are relabelled by a seeded permutation.
    With `n` < 2^scale, samples touching an id >= n are rejected (used by
    the batch mix, where n is not a power of two); `samples` overrides the
    sample count edgefactor * 2^scale."""
    N = 1 << scale
    n_out = N if n is None else int(n)
    samples = edgefactor * N if samples is None else int(samples)
    gd = _rng(seed, device)
    u = torch.zeros(samples, dtype=torch.int64, device=device)
    v = torch.zeros(samples, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    chunk = 1 << 26
    for lvl in range(scale):
        bit = 1 << (scale - 1 - lvl)
        for s0 in range(0, samples, chunk):
            s1 = min(samples, s0 + chunk)
            r = torch.rand(s1 - s0, generator=gd, device=device)
            ubit = r >= ab
            vbit = ((r >= a) & (r < ab)) | (r >= abc)
            u[s0:s1] += ubit.to(torch.int64) * bit
            v[s0:s1] += vbit.to(torch.int64) * bit
            del r, ubit, vbit
    if permute:
        perm = torch.randperm(N, generator=gd, device=device)
        u = perm[u]
        v = perm[v]
    if n_out < N:
        keep = (u < n_out) & (v < n_out)
        u, v = u[keep], v[keep]
    return csr_from_pairs(u, v, n_out)


def complete_graph(n: int, device="cpu"):
    """K_n: every pair adjacent."""
    idx = torch.arange(n, dtype=torch.int64, device=device)
    u = idx.repeat_interleave(n)
    v = idx.repeat(n)
    return csr_from_pairs(u, v, n)


def from_edges(n: int, edges, device="cpu"):
    """CSR from an explicit list of undirected (u, v) pairs."""
    if len(edges) == 0:
        return torch.zeros(n + 1, dtype=torch.int32, device=device), torch.zeros(0, dtype=torch.int32, device=device)
    t = torch.tensor(edges, dtype=torch.int64, device=device)
    return csr_from_pairs(t[:, 0].contiguous(), t[:, 1].contiguous(), n)


def random_pairs(n: int, count: int, seed: int, row_ptr=None, col=None, edge_frac: float = 0.5, device="cpu"):
    """Vertex-pair queries: a fraction drawn from existing edges, the rest
    uniform random pairs (the link-prediction style of Sec. III, Listing 5).
    Returns int32 [count, 2]."""
    g = _rng(seed, device)
    n_edge = int(round(count * edge_frac)) if col is not None and col.numel() > 0 else 0
    out = torch.empty((count, 2), dtype=torch.int32, device=device)
    if n_edge:
        nnz = col.numel()
        j = torch.randint(0, nnz, (n_edge,), generator=g, device=device, dtype=torch.int64)
        src = torch.searchsorted(row_ptr.to(torch.int64), j, right=True) - 1
        out[:n_edge, 0] = src.to(torch.int32)
        out[:n_edge, 1] = col[j]
    if count - n_edge:
        out[n_edge:, 0] = torch.randint(0, n, (count - n_edge,), generator=g, device=device, dtype=torch.int32)
        out[n_edge:, 1] = torch.randint(0, n, (count - n_edge,), generator=g, device=device, dtype=torch.int32)
    return out


def batch_mix(graphs: int, seed: int, log2_n=(8, 16), deg_median: float = 12.0, deg_sigma: float = 0.6,
              deg_range=(4.0, 64.0), device="cpu"):
    """A mix of small graphs of uneven sizes (the batching workload):
    graphs alternate Erdos-Renyi / R-MAT (even index ER, odd R-MAT); each
    has n = floor(2^U(lo, hi)) vertices and a target average degree
    clip(lognormal(ln median, sigma), range). R-MAT graphs use scale
    ceil(log2 n) with ids >= n rejected, drawing enough samples that about
    n * degree / 2 land inside. Returns a list of (row_ptr, col) pairs."""
    rs = np.random.Generator(np.random.PCG64(int(seed)))
    ns = np.floor(2.0 ** rs.uniform(log2_n[0], log2_n[1], graphs)).astype(np.int64)
    degs = np.clip(rs.lognormal(np.log(deg_median), deg_sigma, graphs), deg_range[0], deg_range[1])
    out = []
    for i in range(graphs):
        n, dg = int(ns[i]), float(degs[i])
        gseed = int(seed) * 1_000_003 + i
        if i % 2 == 0:
            out.append(erdos_renyi(n, dg, gseed, device=device))
        else:
            scale = max(1, int(np.ceil(np.log2(n))))
            keep = (n / float(1 << scale)) ** 2
            samples = int(round(n * dg / 2.0 / keep))
            out.append(rmat(scale, 1, gseed, device=device, n=n, samples=samples))
    return out


def block_diagonal(parts):
    """Concatenate graphs into one CSR with global ids: graph i's vertices
    become voff[i] .. voff[i+1]-1. Returns (row_ptr int32, col int32, voff
    int64 numpy [G+1])."""
    ns = [int(rp.numel()) - 1 for rp, _ in parts]
    voff = np.zeros(len(parts) + 1, dtype=np.int64)
    voff[1:] = np.cumsum(ns)
    nnz = [int(cl.numel()) for _, cl in parts]
    eoff = np.zeros(len(parts) + 1, dtype=np.int64)
    eoff[1:] = np.cumsum(nnz)
    if eoff[-1] >= 2**31 or voff[-1] >= 2**31:
        raise ValueError("batch has 2^31 or more vertices or CSR entries")
    device = parts[0][0].device if parts else "cpu"
    row_ptr = torch.empty(int(voff[-1]) + 1, dtype=torch.int32, device=device)
    col = torch.empty(int(eoff[-1]), dtype=torch.int32, device=device)
    for i, (rp, cl) in enumerate(parts):
        row_ptr[voff[i]:voff[i + 1]] = rp[:-1] + int(eoff[i])
        col[eoff[i]:eoff[i + 1]] = cl + int(voff[i])
    row_ptr[-1] = int(eoff[-1])
    return row_ptr, col, voff


def bfs_ball(row_ptr, col, start: int, target_edges: int):
    """Vertices of a breadth-first ball around `start`: whole BFS levels
    while the induced subgraph has fewer than target_edges undirected edges,
    then the shortest prefix of the next level (in BFS discovery order) that
    reaches the target (or the whole component). Host numpy; returns int32
    vertex ids in BFS order (the serving workload's induced-subgraph
    queries)."""
    rp = np.asarray(row_ptr.cpu() if hasattr(row_ptr, "cpu") else row_ptr, dtype=np.int64)
    cl = np.asarray(col.cpu() if hasattr(col, "cpu") else col, dtype=np.int64)
    n = rp.size - 1
    inside = np.zeros(n, dtype=bool)

    def rows(vs):
        lens = rp[vs + 1] - rp[vs]
        idx = np.repeat(rp[vs] - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(int(lens.sum()))
        return cl[idx], np.repeat(np.arange(vs.size), lens)

    def induced_edges(vs):
        mark = np.zeros(n, dtype=bool)
        mark[vs] = True
        nb, _ = rows(vs)
        return int(mark[nb].sum()) // 2

    ball = np.asarray([start], dtype=np.int64)
    inside[start] = True
    frontier = ball
    while frontier.size:
        nb, _ = rows(frontier)
        # next level in discovery order: first occurrence of each new vertex
        new = nb[~inside[nb]]
        _, first = np.unique(new, return_index=True)
        level = new[np.sort(first)]
        if level.size == 0:
            break
        cand = np.concatenate([ball, level])
        if induced_edges(cand) < target_edges:
            inside[level] = True
            ball = cand
            frontier = level
            continue
        lo, hi = 1, level.size  # shortest prefix reaching the target
        while lo < hi:
            mid = (lo + hi) // 2
            if induced_edges(np.concatenate([ball, level[:mid]])) >= target_edges:
                hi = mid
            else:
                lo = mid + 1
        ball = np.concatenate([ball, level[:lo]])
        break
    return ball.astype(np.int32)
