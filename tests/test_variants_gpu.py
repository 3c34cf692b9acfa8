"""GPU parity of the estimator variants (Bloom OR, single-set Bloom on the
AND filter) and of the overlap / total-neighbour similarities, against the
oracle: integer counts (popcount AND and OR) and histograms bit-exact,
per-edge float outputs within 1e-5 relative, double totals within 1e-9."""
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


def _hubs():
    n = 16000
    rp, cl = synth.erdos_renyi(n, 8.0, seed=5)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    g = torch.Generator().manual_seed(5)
    hub = torch.randperm(n, generator=g)[:10000]
    u = torch.cat([src, torch.full((10000,), 7, dtype=torch.int64)])
    v = torch.cat([cl.long(), hub])
    return synth.csr_from_pairs(u, v, n)


GRAPHS = {"er4096": lambda: synth.erdos_renyi(4096, 16.0, seed=1), "rmat12": lambda: synth.rmat(12, 16, seed=7),
          "hubs": _hubs}
_cache = {}


def _graph(name):
    if name not in _cache:
        rp, cl = GRAPHS[name]()
        _cache[name] = (rp.numpy().astype(np.int32), cl.numpy().astype(np.int32))
    return _cache[name]


def _close(got, want, rtol, atol=1e-6):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    bad = np.abs(got - want) > atol + rtol * np.abs(want)
    assert not bad.any(), (np.flatnonzero(bad)[:5], got[bad][:5], want[bad][:5])


# The OR and KMV estimates are d_u + d_v minus a union estimate of similar size,
# each side computed in double: the difference keeps the absolute error of its
# terms, a few ulps of d_u + d_v, while its own magnitude can be far smaller.
# Their float outputs (CN, and total = d_u + d_v - I) are therefore compared with
# a floor of 1e-9 (d_u + d_v) beside the 1e-5 relative bar (reading U).
def _cancel_floor(rp, pu, pv):
    d = np.diff(np.asarray(rp, np.int64)).astype(np.float64)
    return 1e-9 * (d[pu] + d[pv]) + 1e-7


@pytest.mark.parametrize("name", ["er4096", "rmat12", "hubs"])
@pytest.mark.parametrize("est", [6, 7])  # PG_EST_BF_OR, PG_EST_BF_SS
@pytest.mark.parametrize("l,b", [(256, 2), (448, 1), (1024, 4), (192, 2)])
def test_bloom_variants_every_output(pg, name, est, l, b):
    rp, cl = _graph(name)
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    sk = pg.build_bloom(g, l, b, seed=13)
    ref = O.analyze(rp, cl, est, l=l, b=b, seed=13)
    m, n = g.m, g.n
    out = dict(tc=pg.tc_result_buffer(g.device), lcc=torch.empty(n, dtype=torch.float32, device="cuda"),
               tri=torch.empty(n, dtype=torch.float64, device="cuda"),
               edge_cn=torch.empty(m, dtype=torch.float32, device="cuda"),
               edge_jac=torch.empty(m, dtype=torch.float32, device="cuda"),
               edge_count=torch.empty(m, dtype=torch.int32, device="cuda"),
               edge_aux=torch.empty(m, dtype=torch.int32, device="cuda"),
               edge_overlap=torch.empty(m, dtype=torch.float32, device="cuda"),
               edge_total=torch.empty(m, dtype=torch.float32, device="cuda"),
               hist=torch.empty(pg.hist_bins(sk, est), dtype=torch.int64, device="cuda"))
    pg.analyze(g, sk, est, **out)
    tc = pg.read_tc_result(out["tc"])
    cnt = out["edge_count"].cpu().numpy()
    np.testing.assert_array_equal(cnt, ref["counts"]["count"])
    if est == pg.EST_BF_OR:
        np.testing.assert_array_equal(out["edge_aux"].cpu().numpy(), ref["counts"]["union"])
        assert tc["count_sum"] == int(np.sum(ref["counts"]["union"]))
    else:
        assert tc["count_sum"] == int(np.sum(ref["counts"]["count"]))
    np.testing.assert_array_equal(out["hist"].cpu().numpy().view(np.uint64), ref["hist"])
    assert tc["edges"] == ref["m"]
    assert tc["est_tc"] == pytest.approx(ref["tc"], rel=RTOL_F64, abs=1e-9)
    atol = _cancel_floor(rp, ref["eu"], ref["ev"]) if est == pg.EST_BF_OR else 1e-6
    _close(out["edge_cn"].cpu().numpy(), ref["cn"], RTOL_F32, atol)
    _close(out["edge_jac"].cpu().numpy(), ref["jac"], RTOL_F32, 1e-7)
    _close(out["edge_overlap"].cpu().numpy(), ref["overlap"], RTOL_F32, 1e-7)
    _close(out["edge_total"].cpu().numpy(), ref["total"], RTOL_F32, _cancel_floor(rp, ref["eu"], ref["ev"]))
    _close(out["tri"].cpu().numpy(), ref["T"], RTOL_F64, 1e-7)
    _close(out["lcc"].cpu().numpy(), ref["lcc"], RTOL_F32, 1e-6)


@pytest.mark.parametrize("est,kind,kw", [
    (O.EST_EXACT, None, {}),
    (O.EST_BF_AND, "bloom", dict(l=448, b=2)),
    (O.EST_BF_OR, "bloom", dict(l=256, b=2)),
    (O.EST_KH, "khash", dict(k=32)),
    (O.EST_1H, "onehash", dict(k=32)),
    (O.EST_1H_KMV, "onehash", dict(k=32)),
    (O.EST_1H_KMV, "onehash", dict(k=8)),
])
def test_similarity_pairs(pg, est, kind, kw):
    rp, cl = _graph("rmat12")
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    pairs = synth.random_pairs(g.n, 6001, 3, torch.from_numpy(rp), torch.from_numpy(cl)).numpy()
    pairs[:3] = [(-1, 4), (5, g.n + 2), (9, 9)]
    if kind is None:
        sk = None
    elif kind == "bloom":
        sk = pg.build_bloom(g, kw["l"], kw["b"], seed=2)
    else:
        sk = pg.build_minhash(g, pg.SK_KHASH if kind == "khash" else pg.SK_1HASH, kw["k"], seed=2)
    got = pg.similarity_pairs(g, sk, est, torch.from_numpy(pairs).cuda())
    osk = None if kind is None else O.sketch(rp, cl, kind, l=kw.get("l", 256), b=kw.get("b", 2),
                                             k=kw.get("k", 16), seed=2)
    ok = (pairs[:, 0] >= 0) & (pairs[:, 0] < g.n) & (pairs[:, 1] >= 0) & (pairs[:, 1] < g.n)
    pu, pv = pairs[ok, 0], pairs[ok, 1]
    counts = O.pair_counts(rp, cl, est, osk, pu, pv, seed=2)
    e = O.pair_estimates(rp, est, counts, pu, pv, l=kw.get("l", 256), b=kw.get("b", 2), k=kw.get("k", 16))
    want = O.similarities(rp, e, pu, pv)
    floor = _cancel_floor(rp, pu, pv)
    atol = floor if est in (O.EST_BF_OR, O.EST_1H_KMV) else 1e-6
    for nm in ("cn", "jac", "overlap", "total"):
        g_ = got[nm].cpu().numpy()
        _close(g_[ok], want[nm], RTOL_F32, {"cn": atol, "total": floor}.get(nm, 1e-7))
        assert (g_[~ok] == 0.0).all()


def test_variant_pairs_match_edges(pg):
    """The pair path of the OR estimator (generic pass kernel, pairs) and its
    edge path give the same counts on the upper edges."""
    rp, cl = _graph("er4096")
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    sk = pg.build_bloom(g, 512, 2, seed=4)
    eu, ev = O.upper_edges(rp, cl)
    pairs = torch.from_numpy(np.stack([eu, ev], 1).astype(np.int32)).cuda()
    c1, a1, _ = pg.edge_counts(g, sk, pg.EST_BF_OR, pairs, want_aux=True)
    c2, a2, _ = pg.edge_counts(g, sk, pg.EST_BF_OR, None, want_aux=True)
    assert torch.equal(c1, c2) and torch.equal(a1, a2)


@pytest.mark.parametrize("name", ["er4096", "rmat12", "hubs"])
def test_kmv_upper_edges(pg, name):
    """KMV (Sec. IX) on the 1-Hash rows over every upper edge (pairs = NULL) and
    its totals (TC from the 1-Hash histograms and the exact 128-bit sum of the
    real union estimates; per-vertex triangles and LCC), against the oracle."""
    rp, cl = _graph(name)
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    k = 16
    sk = pg.build_minhash(g, pg.SK_1HASH, k, seed=3)
    cn, jac = pg.jaccard_pairs(g, sk, pg.EST_1H_KMV)
    eu, ev = O.upper_edges(rp, cl)
    osk = O.sketch(rp, cl, "onehash", k=k, seed=3)
    counts = O.pair_counts(rp, cl, O.EST_1H_KMV, osk, eu, ev, seed=3)
    e = O.pair_estimates(rp, O.EST_1H_KMV, counts, eu, ev, k=k)
    want = O.similarities(rp, e, eu, ev)
    _close(cn.cpu().numpy(), want["cn"], RTOL_F32, _cancel_floor(rp, eu, ev))
    _close(jac.cpu().numpy(), want["jac"], RTOL_F32, 1e-7)
    c, a, _ = pg.edge_counts(g, sk, pg.EST_1H_KMV, None, want_aux=True)
    np.testing.assert_array_equal(c.cpu().numpy(), counts["count"])
    ref = O.analyze(rp, cl, O.EST_1H_KMV, k=k, seed=3, sk=osk)
    tc = pg.triangle_count(g, sk, pg.EST_1H_KMV)
    assert tc["edges"] == ref["m"] and tc["count_sum"] == int(np.sum(counts["count"]))
    assert tc["est_tc"] == pytest.approx(ref["tc"], rel=RTOL_F64, abs=1e-6)
    lcc, tri, tc2 = pg.clustering(g, sk, pg.EST_1H_KMV)
    assert pg.read_tc_result(tc2)["est_tc"] == tc["est_tc"]  # the 128-bit sum does not depend on order
    # per-vertex sums of estimates of both signs: double additions in any order keep
    # the absolute error within a few ulps of the sum of the magnitudes
    mag = np.zeros(g.n)
    np.add.at(mag, eu, np.abs(e))
    np.add.at(mag, ev, np.abs(e))
    _close(tri.cpu().numpy(), ref["T"], RTOL_F64, 1e-12 * mag + 1e-12)
    _close(lcc.cpu().numpy(), ref["lcc"], RTOL_F32, 1e-7)
