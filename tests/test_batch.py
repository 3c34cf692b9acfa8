"""Batched analysis of many small graphs (pg_batch_*).

CPU tests: the autotuner's rules and the argument checks, which run on the
host. GPU tests: every graph's triangle count, edge totals and per-vertex
LCC from one batched run (eager, captured and replayed) equal those of the
single-graph entry points on the same graph, and the oracle's on a few.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2208_11469_gb300 import synth

RTOL_F32 = 1e-5
RTOL_F64 = 1e-9


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


# ------------------------------------------------------------------ host only
def test_autotune_bits_follow_the_storage_budget(pg):
    """bits = the largest power of two in [64, 1024] not above the budget's
    bits per vertex, s * (4(n+1) + 4 nnz) * 8 / n (storage budget, Sec. V-A)."""
    n = np.array([256, 1000, 4096, 50000, 65536, 300], dtype=np.int32)
    nnz = np.array([1024, 12000, 65536, 3_000_000, 640_000, 300 * 299], dtype=np.int64)
    for s in (0.1, 0.25, 0.5, 1.0):
        cfg = pg.batch_autotune(n, nnz, s)
        for i in range(len(n)):
            per_vertex = s * (4.0 * (n[i] + 1) + 4.0 * nnz[i]) * 8.0 / n[i]
            want = 64
            while want * 2 <= per_vertex and want < 1024:
                want *= 2
            assert cfg[i][0] == want, (s, i, cfg[i], per_vertex)
            assert cfg[i][1] in (1, 2, 4)


def test_autotune_hash_count_falls_as_filters_fill(pg):
    """The model trades the AND estimator's variance (the Prop. 4.1 bound,
    which falls as b grows) against the bias from collisions of the
    elements the two sets do not share (which grows with b and with the
    degree). At a fixed filter length, while rows leave most bits zero,
    denser neighbourhoods must therefore get no more hash functions than
    sparser ones; rows with nothing to collide get the most."""
    n = np.full(8, 4096, dtype=np.int32)
    degs = np.array([1, 2, 3, 4, 6, 8, 16, 32], dtype=np.int64)
    cfg = pg.batch_autotune(n, n.astype(np.int64) * degs, 0.001)  # tiny budget: every graph at 64 bits
    assert all(c[0] == 64 for c in cfg)
    bs = [c[1] for c in cfg]
    assert bs == sorted(bs, reverse=True), bs
    assert bs[0] == 4 and bs[-1] == 1
    cfg = pg.batch_autotune(np.array([4096], np.int32), np.array([4096], np.int64), 100.0)
    assert cfg[0] == (1024, 4)  # degree 1: no private elements, variance only


def _csr_stub(n, nnz):
    from paper_2208_11469_gb300 import pg as _pg
    return _pg.Csr(None, None, n, nnz)


def test_workspace_rejects_bad_batches(pg):
    L = pg.lib()
    voff = np.array([0, 10, 20, 30], dtype=np.int32)
    c = _csr_stub(30, 100)

    def ws(cfgs):
        arr = (pg.BatchConfig * 3)(*[pg.BatchConfig(b, h, 0, 0) for b, h in cfgs])
        return L.pg_batch_workspace_bytes(ctypes.byref(c), 3, voff.ctypes.data_as(ctypes.c_void_p), arr)

    assert ws([(256, 2), (256, 2), (512, 1)]) > 0
    assert ws([(256, 2), (512, 1), (256, 2)]) == 0
    assert "contiguous" in L.pg_last_error().decode()
    assert ws([(256, 2), (300, 2), (300, 2)]) == 0
    assert "300" in L.pg_last_error().decode()
    assert ws([(256, 0), (256, 0), (256, 0)]) == 0
    arr = (pg.BatchConfig * 3)(*[pg.BatchConfig(256, 2, v, 0) for v in (1, 1025, 1)])
    assert L.pg_batch_workspace_bytes(ctypes.byref(c), 3, voff.ctypes.data_as(ctypes.c_void_p), arr) == 0
    assert "variant" in L.pg_last_error().decode()
    big = _csr_stub(30, 2**31 - 40)
    arr = (pg.BatchConfig * 3)(*[pg.BatchConfig(256, 2, 0, 0)] * 3)
    assert L.pg_batch_workspace_bytes(ctypes.byref(big), 3, voff.ctypes.data_as(ctypes.c_void_p), arr) == 0
    assert "nnz" in L.pg_last_error().decode()
    bad = np.array([0, 20, 10, 30], dtype=np.int32)
    arr = (pg.BatchConfig * 3)(*[pg.BatchConfig(256, 2, 0, 0)] * 3)
    assert L.pg_batch_workspace_bytes(ctypes.byref(c), 3, bad.ctypes.data_as(ctypes.c_void_p), arr) == 0


def test_workspace_grows_with_the_sketches(pg):
    L = pg.lib()
    voff = np.array([0, 1000, 3000], dtype=np.int32)
    c = _csr_stub(3000, 40000)

    def ws(bits):
        arr = (pg.BatchConfig * 2)(pg.BatchConfig(bits, 2, 0, 0), pg.BatchConfig(1024, 2, 0, 0))
        return L.pg_batch_workspace_bytes(ctypes.byref(c), 2, voff.ctypes.data_as(ctypes.c_void_p), arr)

    a, b = ws(64), ws(512)
    assert b - a >= 1000 * (64 - 16) - 256  # 16 B rows -> 64 B rows for the first graph
    assert a >= 3000 * 16 + 8 * (65 + 1025)


# ------------------------------------------------------------------- GPU
CONFIGS = [(64, 1), (128, 2), (256, 2), (512, 4), (1024, 1), (256, 1)]


def _mix():
    """A small mix of uneven graphs, plus the cases the batch must carry
    through: a graph without edges, a one-vertex graph, an empty graph, and a
    graph with a hub above the one-warp Bloom builder's threshold."""
    parts = synth.batch_mix(18, seed=11, log2_n=(6, 11))
    parts.append(synth.from_edges(7, []))
    parts.append(synth.from_edges(1, []))
    parts.append((torch.zeros(1, dtype=torch.int32), torch.zeros(0, dtype=torch.int32)))
    n = 12000
    rp, cl = synth.erdos_renyi(n, 6.0, seed=4)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    hub = torch.randperm(n, generator=torch.Generator().manual_seed(2))[:9500]
    u = torch.cat([src, torch.zeros(9500, dtype=torch.int64)])
    v = torch.cat([cl.long(), hub])
    parts.append(synth.csr_from_pairs(u.long(), v.long(), n))
    return parts


def _assign(parts):
    """Configs cycling through the widths, graphs reordered so that equal
    configurations are contiguous."""
    cfg = [CONFIGS[i % len(CONFIGS)] for i in range(len(parts))]
    order = sorted(range(len(parts)), key=lambda i: (CONFIGS.index(cfg[i]), i))
    return [parts[i] for i in order], [cfg[i] for i in order]


def _single(pg, rp, cl, bits, b, seed):
    n = rp.numel() - 1
    if n == 0:
        return dict(edges=0, count_sum=0, est_tc=0.0, est_tc_alt=0.0), np.zeros(0, np.float32)
    g = pg.graph(rp.cuda(), cl.cuda())
    sk = pg.build_bloom(g, bits, b, seed=seed)
    lcc, _, tc = pg.clustering(g, sk, pg.EST_BF_AND, want_tri=False)
    return pg.read_tc_result(tc), lcc.cpu().numpy()


@pytest.mark.gpu
def test_batch_matches_single_graph_calls(pg):
    parts, cfg = _assign(_mix())
    rp, cl, voff = synth.block_diagonal(parts)
    seed = 5
    batch = pg.Batch(pg.graph(rp.cuda(), cl.cuda(), build_index=False), voff, cfg, seed=seed, want_tri=True)
    want = [_single(pg, p[0], p[1], c[0], c[1], seed) for p, c in zip(parts, cfg)]
    side = torch.cuda.Stream()
    runs = [("eager", None), ("capture", side), ("replay", side)]
    for label, stream in runs:
        batch.lcc.fill_(-1.0)
        batch.tc.fill_(0xAB)
        if stream is None:
            batch.run()
        else:
            with torch.cuda.stream(stream):
                batch.run()
            stream.synchronize()
        torch.cuda.synchronize()
        got = batch.results()
        lcc = batch.lcc.cpu().numpy()
        tri = batch.tri.cpu().numpy()
        for i, ((w, wl), g) in enumerate(zip(want, got)):
            assert g["edges"] == w["edges"] and g["count_sum"] == w["count_sum"], (label, i, cfg[i])
            assert g["est_tc"] == pytest.approx(w["est_tc"], rel=RTOL_F64, abs=1e-12), (label, i)
            assert g["est_tc_alt"] == pytest.approx(w["est_tc_alt"], rel=RTOL_F64, abs=1e-12), (label, i)
            gl = lcc[voff[i]:voff[i + 1]]
            np.testing.assert_allclose(gl, wl, rtol=RTOL_F32, atol=1e-6, err_msg=f"{label} graph {i}")
        # per-vertex triangles sum to three times each graph's estimate
        for i in range(len(parts)):
            assert tri[voff[i]:voff[i + 1]].sum() == pytest.approx(3 * got[i]["est_tc"], rel=1e-9, abs=1e-9)
    assert all(v in (1, 4, 16) for v in batch.variants)
    batch.close()


@pytest.mark.gpu
@pytest.mark.parametrize("chunk,own_stream", [(1, True), (5000, True), (1 << 30, True), (5000, False)])
def test_run_host_matches_device_run(pg, chunk, own_stream):
    """pg_batch_run_host uploads the union CSR in chunks of whole graphs while
    it works on the chunks already copied: after it, the device CSR equals the
    host one and every output is bit-identical to a run on that CSR. The host
    CSR differs from the one the batch was created on (inside each graph the
    column ids are mapped by a permutation of its vertices), so a run that
    did not upload would be caught."""
    parts, cfg = _assign(_mix())
    rp, cl, voff = synth.block_diagonal(parts)
    gen = torch.Generator().manual_seed(7)
    perm = torch.arange(rp.numel() - 1, dtype=torch.int64)
    for i in range(len(voff) - 1):
        a, b = int(voff[i]), int(voff[i + 1])
        if b > a:
            perm[a:b] = a + torch.randperm(b - a, generator=gen)
    cl2 = perm[cl.long()].to(torch.int32)
    dev_rp, dev_cl = rp.cuda(), cl.cuda()
    batch = pg.Batch(pg.graph(dev_rp, dev_cl, build_index=False), voff, cfg, seed=5, want_tri=True)
    dev_cl.copy_(cl2.cuda())
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        batch.run()
    side.synchronize()
    want = (batch.results(), batch.lcc.cpu().numpy().copy(), batch.tri.cpu().numpy().copy())
    dev_cl.copy_(cl.cuda())
    batch.lcc.fill_(-1.0)
    batch.tri.fill_(-1.0)
    torch.cuda.synchronize()
    cs = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
    batch.run_host(rp.pin_memory(), cl2.pin_memory(), chunk_entries=chunk, copy_stream=cs)
    torch.cuda.synchronize()
    assert torch.equal(dev_cl.cpu(), cl2) and torch.equal(dev_rp.cpu(), rp)
    assert batch.results() == want[0]
    np.testing.assert_array_equal(batch.lcc.cpu().numpy(), want[1])
    np.testing.assert_array_equal(batch.tri.cpu().numpy(), want[2])
    batch.close()


@pytest.mark.gpu
def test_64_bit_build_with_hub_rows(pg):
    """The 64-bit buckets use their own builder (one warp walks 32 rows'
    entries, so a hub row is walked by one warp): a graph with a 9500-entry
    hub row and graphs with isolated vertices give the single-graph results."""
    n = 12000
    rp, cl = synth.erdos_renyi(n, 6.0, seed=4)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    hub = torch.randperm(n, generator=torch.Generator().manual_seed(2))[:9500]
    u = torch.cat([src, torch.full((9500,), 77, dtype=torch.int64)])
    v = torch.cat([cl.long(), hub])
    parts = [synth.csr_from_pairs(u.long(), v.long(), n), synth.from_edges(40, [(0, 1), (1, 2), (0, 2)]),
             synth.erdos_renyi(300, 4.0, seed=8)]
    cfg = [(64, 2)] * len(parts)
    rp_u, cl_u, voff = synth.block_diagonal(parts)
    batch = pg.Batch(pg.graph(rp_u.cuda(), cl_u.cuda(), build_index=False), voff, cfg, seed=3)
    batch.run()
    torch.cuda.synchronize()
    got = batch.results()
    lcc = batch.lcc.cpu().numpy()
    for i, (p_, c) in enumerate(zip(parts, cfg)):
        w, wl = _single(pg, p_[0], p_[1], c[0], c[1], 3)
        assert (got[i]["edges"], got[i]["count_sum"]) == (w["edges"], w["count_sum"]), i
        assert got[i]["est_tc"] == pytest.approx(w["est_tc"], rel=RTOL_F64, abs=1e-12)
        np.testing.assert_allclose(lcc[voff[i]:voff[i + 1]], wl, rtol=RTOL_F32, atol=1e-6)
    batch.close()


@pytest.mark.gpu
def test_batch_against_oracle(pg):
    from oracle import oracle as O
    # every bucket width, the 64-bit one (flat-walk build and pull pass) included, and a
    # 64-bit graph with a 9 500-neighbour hub row
    parts = synth.batch_mix(9, seed=3, log2_n=(7, 10))
    n_h = 12000
    rp_h, cl_h = synth.erdos_renyi(n_h, 6.0, seed=4)
    src = torch.repeat_interleave(torch.arange(n_h), (rp_h[1:] - rp_h[:-1]).long())
    hub = torch.randperm(n_h, generator=torch.Generator().manual_seed(2))[:9500]
    hub_graph = synth.csr_from_pairs(torch.cat([src, torch.full((9500,), 77, dtype=torch.int64)]),
                                     torch.cat([cl_h.long(), hub]), n_h)
    parts = parts[:6] + [hub_graph] + parts[6:]
    # graphs of one (bits, b) bucket are contiguous
    cfg = [(256, 2), (256, 2), (512, 1), (128, 4), (64, 1), (64, 2), (64, 2), (64, 4), (1024, 2), (128, 1)]
    rp, cl, voff = synth.block_diagonal(parts)
    batch = pg.Batch(pg.graph(rp.cuda(), cl.cuda(), build_index=False), voff, cfg, seed=9, want_tri=True)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        batch.run()
    side.synchronize()
    got = batch.results()
    lcc = batch.lcc.cpu().numpy()
    tri = batch.tri.cpu().numpy()
    for i, ((prp, pcl), (bits, b)) in enumerate(zip(parts, cfg)):
        ref = O.analyze(prp.numpy(), pcl.numpy(), O.EST_BF_AND, l=bits, b=b, seed=9)
        assert got[i]["edges"] == ref["m"], i
        assert got[i]["count_sum"] == int(np.sum(ref["counts"]["count"])), i
        assert got[i]["est_tc"] == pytest.approx(ref["tc"], rel=RTOL_F64), i
        np.testing.assert_allclose(lcc[voff[i]:voff[i + 1]], ref["lcc"], rtol=RTOL_F32, atol=1e-6)
        np.testing.assert_allclose(tri[voff[i]:voff[i + 1]], ref["T"], rtol=RTOL_F64, atol=1e-9)
    batch.close()


@pytest.mark.gpu
def test_batch_variants_give_identical_results(pg):
    """The per-vertex sums are exact fixed-point sums, so every work mapping
    (variant = 32-vertex groups per warp chunk) gives bit-identical per-graph
    totals, LCC and per-vertex triangles, and so do repeated runs."""
    parts = synth.batch_mix(6, seed=21, log2_n=(9, 12))
    rp, cl, voff = synth.block_diagonal(parts)
    g = pg.graph(rp.cuda(), cl.cuda(), build_index=False)
    for bits in (64, 128, 256, 512, 1024):
        res = []
        for var in (1, 3, 16, 1):
            bt = pg.Batch(g, voff, [(bits, 2, var)] * len(parts), seed=1, want_tri=True)
            bt.run()
            torch.cuda.synchronize()
            res.append(([(r["edges"], r["count_sum"], r["est_tc"]) for r in bt.results()], bt.lcc.cpu().numpy(),
                        bt.tri.cpu().numpy()))
            assert bt.variants == [var] * len(parts)
            bt.close()
        for other in res[1:]:
            assert other[0] == res[0][0], bits
            np.testing.assert_array_equal(other[1], res[0][1])
            np.testing.assert_array_equal(other[2], res[0][2])
