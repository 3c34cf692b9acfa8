"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded graphs.

Bar: bit-exact sketches, per-edge integer
counts and histograms; 1e-5 relative on per-edge float32 estimates,
Jaccard and LCC; 1e-9 relative on double totals and per-vertex triangles."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL_F32 = 1e-5
RTOL_F64 = 1e-9


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


def _np(t):
    return t.cpu().numpy()


def _graph(pg, rp, cl):
    return pg.graph(rp.to(torch.int32).cuda(), cl.to(torch.int32).cuda())


def _hub_graph(seed=3):
    """ER background plus three hubs whose degrees exceed every builder's
    one-warp threshold (8192 Bloom, 2048 k-Hash, 4096 1-Hash)."""
    n = 24000
    rp, cl = synth.erdos_renyi(n, 8.0, seed=seed)
    g = torch.Generator().manual_seed(seed)
    u = [torch.repeat_interleave(torch.tensor([0]), 9000), torch.repeat_interleave(torch.tensor([1]), 12500),
         torch.repeat_interleave(torch.tensor([2]), 20000)]
    v = [torch.randperm(n, generator=g)[:9000], torch.randperm(n, generator=g)[:12500],
         torch.randperm(n, generator=g)[:20000]]
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    u = torch.cat([src] + u).long()
    v = torch.cat([cl.long()] + v).long()
    return synth.csr_from_pairs(u, v, n)


GRAPHS = {
    "er4096": lambda: synth.erdos_renyi(4096, 16.0, seed=1),
    "rmat12": lambda: synth.rmat(12, 16, seed=7),
    "hubs": _hub_graph,
}
_cache = {}


def graph_np(name):
    if name not in _cache:
        rp, cl = GRAPHS[name]()
        _cache[name] = (rp.numpy().astype(np.int32), cl.numpy().astype(np.int32))
    return _cache[name]


def _dev(pg, name):
    rp, cl = graph_np(name)
    return _graph(pg, torch.from_numpy(rp), torch.from_numpy(cl)), rp, cl


# ------------------------------------------------------------------ sketches

@pytest.mark.parametrize("name", ["er4096", "rmat12", "hubs"])
@pytest.mark.parametrize("bits,b", [(256, 2), (64, 1), (192, 4), (448, 2), (960, 2), (1024, 3)])
def test_bloom_sketch_bit_exact(pg, name, bits, b):
    g, rp, cl = _dev(pg, name)
    sk = pg.build_bloom(g, bits, b, seed=11)
    words = sk.stride // 8
    got = _np(sk.data.view(torch.int64)).view(np.uint64).reshape(g.n, words)
    want = O.bloom_pack(O.bloom_bits(rp, cl, bits, b, 11), words)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name", ["er4096", "rmat12", "hubs"])
@pytest.mark.parametrize("k", [16, 64, 7, 32, 100])
def test_khash_sketch_bit_exact(pg, name, k):
    if name == "hubs" and k == 100:
        pytest.skip("covered by k=64")
    g, rp, cl = _dev(pg, name)
    sk = pg.build_minhash(g, pg.SK_KHASH, k, seed=5)
    got = _np(sk.data.view(torch.int32)).view(np.uint32).reshape(g.n, sk.stride // 4)[:, :k]
    want = O.khash_values(O.khash(rp, cl, k, 5), 5)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name", ["er4096", "rmat12", "hubs"])
@pytest.mark.parametrize("k", [32, 8, 19])
def test_onehash_sketch_bit_exact(pg, name, k):
    g, rp, cl = _dev(pg, name)
    sk = pg.build_minhash(g, pg.SK_1HASH, k, seed=9)
    got = _np(sk.data.view(torch.int32)).view(np.uint32).reshape(g.n, sk.stride // 4)[:, :k]
    want = O.onehash_values(O.onehash(rp, cl, k, 9), 9)
    assert np.array_equal(got, want)


# --------------------------------------------------- counts and estimates

CASES = [
    ("er4096", O.EST_BF_AND, dict(l=256, b=2)),
    ("er4096", O.EST_BF_L, dict(l=256, b=2)),
    ("er4096", O.EST_KH, dict(k=16)),
    ("er4096", O.EST_1H, dict(k=32)),
    ("er4096", O.EST_1H_LITERAL, dict(k=32)),
    ("rmat12", O.EST_BF_AND, dict(l=192, b=1)),
    ("rmat12", O.EST_BF_AND, dict(l=448, b=4)),
    ("rmat12", O.EST_KH, dict(k=64)),
    ("rmat12", O.EST_1H, dict(k=32)),
    ("hubs", O.EST_BF_AND, dict(l=960, b=2)),
    ("hubs", O.EST_KH, dict(k=64)),
    ("hubs", O.EST_1H, dict(k=16)),
]


def _sketch(pg, g, est, kw, seed):
    if est in (O.EST_BF_AND, O.EST_BF_L):
        return pg.build_bloom(g, kw["l"], kw["b"], seed=seed)
    if est == O.EST_KH:
        return pg.build_minhash(g, pg.SK_KHASH, kw["k"], seed=seed)
    if est in (O.EST_1H, O.EST_1H_LITERAL):
        return pg.build_minhash(g, pg.SK_1HASH, kw["k"], seed=seed)
    return None


def _oracle_hist(r, est, kw, d):
    c = np.asarray(r["counts"]["count"], np.int64)
    if est in (O.EST_BF_AND, O.EST_BF_L):
        return np.bincount(c, minlength=kw["l"] + 1).astype(np.uint64)
    if est == O.EST_KH:
        return np.concatenate([r["hist"], r["hist_deg"]])
    k = kw["k"]
    hk = k + 1
    K, lit = r["counts"]["K"].astype(np.int64), r["counts"]["c_lit"].astype(np.int64)
    ds = (d[r["eu"]] + d[r["ev"]]).astype(np.int64)
    h = np.zeros(2 * hk * hk + 2 * hk, np.int64)
    np.add.at(h, K * hk + c, 1)
    np.add.at(h, hk * hk + K * hk + c, ds)
    np.add.at(h, 2 * hk * hk + lit, 1)
    np.add.at(h, 2 * hk * hk + hk + lit, ds)
    return h.astype(np.uint64)


@pytest.mark.parametrize("name,est,kw", CASES)
def test_edge_counts_histogram_tc_lcc_jaccard(pg, name, est, kw):
    seed = 21
    g, rp, cl = _dev(pg, name)
    sk = _sketch(pg, g, est, kw, seed)
    r = O.analyze(rp, cl, est, seed=seed, **kw)
    d = O.degrees(rp)
    assert g.m == r["m"]
    # per-edge integer counts (upper-edge order), bit-exact
    cnt, aux, hist = pg.edge_counts(g, sk, est, want_aux=est in (O.EST_1H, O.EST_1H_LITERAL), want_hist=True)
    want_cnt = r["counts"]["c_lit"] if est == O.EST_1H_LITERAL else r["counts"]["count"]
    assert np.array_equal(_np(cnt), np.asarray(want_cnt, np.int32))
    if aux is not None:
        a = _np(aux)
        assert np.array_equal(a & 0xFFFF, r["counts"]["K"]) and np.array_equal(a >> 16, r["counts"]["c_lit"])
    assert np.array_equal(_np(hist).view(np.uint64), _oracle_hist(r, est, kw, d))
    # graph total and its companion estimate
    tc = pg.triangle_count(g, sk, est)
    assert tc["edges"] == r["m"]
    assert tc["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64, abs=1e-12)
    if est in (O.EST_BF_AND, O.EST_BF_L):
        other = O.EST_BF_L if est == O.EST_BF_AND else O.EST_BF_AND
        r2 = O.analyze(rp, cl, other, seed=seed, sk=r["sketch"], **kw)
        assert tc["est_tc_alt"] == pytest.approx(r2["tc"], rel=RTOL_F64, abs=1e-12)
        assert tc["count_sum"] == int(np.sum(r["counts"]["count"]))
    # clustering (same pass also gives TC)
    lcc, tri, tcb = pg.clustering(g, sk, est)
    assert np.allclose(_np(tri), r["T"], rtol=RTOL_F64, atol=1e-9)
    assert np.allclose(_np(lcc), r["lcc"], rtol=RTOL_F32, atol=1e-7)
    assert pg.read_tc_result(tcb)["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64, abs=1e-12)
    # per-edge common neighbours and Jaccard
    cn, jac = pg.jaccard_pairs(g, sk, est)
    assert np.allclose(_np(cn), r["cn"].astype(np.float32), rtol=RTOL_F32, atol=1e-6)
    assert np.allclose(_np(jac), r["jac"], rtol=RTOL_F32, atol=1e-7)


@pytest.mark.parametrize("name", ["er4096", "hubs"])
def test_exact_path(pg, name):
    g, rp, cl = _dev(pg, name)
    r = O.analyze(rp, cl, O.EST_EXACT)
    tc = pg.triangle_count(g, None, O.EST_EXACT)
    assert tc["exact_tc"] == r["tc_exact"]
    assert tc["edges"] == r["m"] and tc["count_sum"] == 3 * r["tc_exact"]
    lcc, tri, tcb = pg.clustering(g, None, O.EST_EXACT)
    assert np.array_equal(_np(tri), r["T"])
    assert np.allclose(_np(lcc), r["lcc"], rtol=RTOL_F32, atol=1e-7)
    assert pg.read_tc_result(tcb)["exact_tc"] == r["tc_exact"]
    cnt, _, _ = pg.edge_counts(g, None, O.EST_EXACT)
    assert np.array_equal(_np(cnt), r["counts"]["count"].astype(np.int32))
    cn, jac = pg.jaccard_pairs(g, None, O.EST_EXACT)
    assert np.allclose(_np(jac), r["jac"], rtol=RTOL_F32, atol=1e-7)


# -------------------------------------------------------------------- pairs

@pytest.mark.parametrize("est,kw", [(O.EST_BF_AND, dict(l=256, b=2)), (O.EST_KH, dict(k=32)),
                                    (O.EST_1H, dict(k=32)), (O.EST_EXACT, {})])
def test_pairs(pg, est, kw):
    g, rp, cl = _dev(pg, "hubs")
    pairs = synth.random_pairs(g.n, 5003, seed=4, row_ptr=torch.from_numpy(rp), col=torch.from_numpy(cl))
    pairs[:7, 1] = pairs[:7, 0]          # u == v
    pairs[7:9, 0] = int(np.flatnonzero(O.degrees(rp) == 0)[0]) if (O.degrees(rp) == 0).any() else 5
    pu, pv = pairs[:, 0].numpy(), pairs[:, 1].numpy()
    sk = _sketch(pg, g, est, kw, 33)
    osk = O.sketch(rp, cl, {O.EST_BF_AND: "bloom", O.EST_KH: "khash", O.EST_1H: "onehash"}[est], seed=33,
                   **kw) if est != O.EST_EXACT else None
    cnts = O.pair_counts(rp, cl, est, osk, pu, pv, seed=33)
    e = O.pair_estimates(rp, est, cnts, pu, pv, **kw)
    cn_o, jac_o = O.jaccard_and_cn(rp, e, pu, pv)
    dp = pairs.cuda()
    cnt, _, _ = pg.edge_counts(g, sk, est, dp)
    assert np.array_equal(_np(cnt), np.asarray(cnts["count"], np.int32))
    cn, jac = pg.jaccard_pairs(g, sk, est, dp)
    assert np.allclose(_np(cn), cn_o.astype(np.float32), rtol=RTOL_F32, atol=1e-6)
    assert np.allclose(_np(jac), jac_o, rtol=RTOL_F32, atol=1e-7)


# --------------------------------------------------------------- edge cases

@pytest.mark.parametrize("edges,n", [([], 0), ([], 6), ([(0, 1)], 2), ([(0, 1), (1, 2), (0, 2)], 5),
                                     ([(i, j) for i in range(7) for j in range(i + 1, 7)], 7)])
def test_degenerate_graphs(pg, edges, n):
    rp, cl = synth.from_edges(n, edges)
    rp_np, cl_np = rp.numpy().astype(np.int32), cl.numpy().astype(np.int32)
    g = _graph(pg, rp, cl)
    for est, kw in [(O.EST_BF_AND, dict(l=64, b=2)), (O.EST_KH, dict(k=8)), (O.EST_1H, dict(k=4)),
                    (O.EST_EXACT, {})]:
        r = O.analyze(rp_np, cl_np, est, seed=2, **kw)
        sk = _sketch(pg, g, est, kw, 2)
        tc = pg.triangle_count(g, sk, est)
        assert tc["edges"] == r["m"]
        assert tc["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64, abs=1e-12)
        if est == O.EST_EXACT:
            assert tc["exact_tc"] == r["tc_exact"]
        lcc, tri, _ = pg.clustering(g, sk, est)
        assert np.allclose(_np(tri), r["T"], rtol=RTOL_F64, atol=1e-12)
        assert np.allclose(_np(lcc), r["lcc"], rtol=RTOL_F32, atol=1e-7)


def test_padded_stride_and_row_padding(pg):
    """A stride wider than the payload: Bloom padding words are written as
    zero and never change a count; MinHash rows ignore their padding."""
    g, rp, cl = _dev(pg, "er4096")
    sk = pg.build_bloom(g, 192, 2, seed=4, stride=64)
    words = _np(sk.data.view(torch.int64)).view(np.uint64).reshape(g.n, 8)
    assert np.array_equal(words[:, :3], O.bloom_pack(O.bloom_bits(rp, cl, 192, 2, 4), 3))
    assert not words[:, 3:].any()
    r = O.analyze(rp, cl, O.EST_BF_AND, l=192, b=2, seed=4)
    cnt, _, _ = pg.edge_counts(g, sk, O.EST_BF_AND)
    assert np.array_equal(_np(cnt), r["counts"]["count"])
    skk = pg.alloc_sketch(g, pg.SK_KHASH, k=30, seed=4, stride=256)
    skk.data.fill_(0x5A)
    pg.build_minhash(g, pg.SK_KHASH, 30, seed=4, out=skk)
    rk = O.analyze(rp, cl, O.EST_KH, k=30, seed=4)
    cnt, _, _ = pg.edge_counts(g, skk, O.EST_KH)
    assert np.array_equal(_np(cnt), rk["counts"]["count"])


def test_validate_csr_reports_malformed_graphs(pg):
    rp, cl = synth.erdos_renyi(300, 6.0, seed=5)
    g = _graph(pg, rp, cl)
    assert pg.validate_csr(g) == ("ok", 0)
    bad = cl.clone()
    bad[10] = 300                                   # out of range (also leaves an asymmetric pair)
    assert pg.validate_csr(_graph(pg, rp, bad)) == ("out_of_range", 10)
    bad = cl.clone()
    r0 = int(rp[5])
    bad[r0] = 5                                     # self loop in row 5
    code = pg.validate_csr(_graph(pg, rp, bad))[0]
    assert code in ("self_loop", "unsorted", "asymmetric")
    bad = cl.clone()
    a, b_ = int(rp[7]), int(rp[8])
    if b_ - a >= 2:
        bad[a], bad[a + 1] = cl[a + 1], cl[a]       # unsorted row
        assert pg.validate_csr(_graph(pg, rp, bad), check_symmetry=False)[0] == "unsorted"
    # drop one direction of an edge: asymmetric
    u = 9
    j = int(rp[u])
    v = int(cl[j])
    keep = torch.ones(cl.numel(), dtype=torch.bool)
    keep[j] = False
    rp2 = rp.clone()
    rp2[u + 1:] -= 1
    assert pg.validate_csr(_graph(pg, rp2, cl[keep]))[0] == "asymmetric"
    rp3 = rp.clone()
    rp3[-1] += 1
    assert pg.validate_csr(pg.Graph(rp3.cuda(), cl.cuda()))[0] == "bad_row_ptr"


def test_sketch_file_round_trip(pg, tmp_path):
    """A saved sketch loads back bit for bit and gives the same counts; a file
    whose descriptor differs from the target is refused."""
    g, rp, cl = _dev(pg, "rmat12")
    for sk in (pg.build_bloom(g, 448, 2, seed=3), pg.build_minhash(g, pg.SK_KHASH, 64, seed=3),
               pg.build_minhash(g, pg.SK_1HASH, 32, seed=3)):
        path = str(tmp_path / f"s{sk.kind}.pgs")
        pg.sketch_save(sk, path)
        back = pg.sketch_load(path)
        assert (back.kind, back.bits, back.b, back.k, back.seed, back.n, back.stride) == \
            (sk.kind, sk.bits, sk.b, sk.k, sk.seed, sk.n, sk.stride)
        assert torch.equal(back.data[: g.n * sk.stride], sk.data[: g.n * sk.stride])
        est = {pg.SK_BLOOM: pg.EST_BF_AND, pg.SK_KHASH: pg.EST_KH, pg.SK_1HASH: pg.EST_1H}[sk.kind]
        assert pg.triangle_count(g, back, est) == pg.triangle_count(g, sk, est)
    other = pg.alloc_sketch(g, pg.SK_BLOOM, bits=448, b=1, seed=3)
    d = other.desc()
    import ctypes
    assert pg.lib().pg_sketch_load(ctypes.byref(d), str(tmp_path / f"s{pg.SK_BLOOM}.pgs").encode(), None) == -1
